// Host runtime behind the C ABI of include/tpmc.h: contexts, resident meshes,
// memory admission, query set-up, launches and result read-back.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "runtime.h"

namespace tpmc {

thread_local std::string g_last_error;

tpmc_status fail(tpmc_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

tpmc_status cuda_fail(cudaError_t e, const char* where) {
  return fail(TPMC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------ allocation
tpmc_status Ctx::alloc(void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) return TPMC_OK;
  if (used + bytes > budget)
    return fail(TPMC_ENOMEM, std::string(what) + ": memory budget exceeded (" + std::to_string(used + bytes) +
                                 " > " + std::to_string(budget) + " bytes)");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(TPMC_ENOMEM, std::string(what) + ": cudaMalloc: " + cudaGetErrorString(e));
  }
  sizes[*p] = bytes;
  used += bytes;
  ++n_allocs;
  return TPMC_OK;
}

void Ctx::release(void* p) {
  if (!p) return;
  auto it = sizes.find(p);
  if (it != sizes.end()) {
    used -= it->second;
    sizes.erase(it);
  }
  cudaFree(p);
}

tpmc_status Ctx::grow(Scratch& s, size_t bytes, const char* what) {
  if (s.cap >= bytes) return TPMC_OK;
  release(s.ptr);
  s.ptr = nullptr;
  s.cap = 0;
  size_t want = std::max(bytes, (size_t)256);
  tpmc_status st = alloc(&s.ptr, want, what);
  if (st == TPMC_OK) s.cap = want;
  return st;
}

// ---------------------------------------------------------------- params
tpmc_status validate_params(const tpmc_params* p) {
  if (!p) return fail(TPMC_EINVAL, "params is NULL");
  const double pos[] = {p->n, p->T_inf, p->m, p->V, p->T_W, p->A_ref};
  const char* names[] = {"n", "T_inf", "m", "V", "T_W", "A_ref"};
  for (int i = 0; i < 6; ++i)
    if (!(std::isfinite(pos[i]) && pos[i] > 0.0)) return fail(TPMC_EINVAL, std::string(names[i]) + " must be finite and > 0");
  if (!(p->eps_diffuse >= 0.0 && p->eps_diffuse <= 1.0)) return fail(TPMC_EINVAL, "eps_diffuse must be in [0, 1]");
  const double dn = std::sqrt(p->dir[0] * p->dir[0] + p->dir[1] * p->dir[1] + p->dir[2] * p->dir[2]);
  if (!(std::isfinite(dn) && dn > 0.0)) return fail(TPMC_EINVAL, "dir must be finite and non-zero");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(p->ref_point[i]) || !std::isfinite(p->center[i])) return fail(TPMC_EINVAL, "non-finite point");
  if (!std::isfinite(p->r_cv)) return fail(TPMC_EINVAL, "r_cv must be finite");
  // the trace kernel keeps a particle's hit count in 24 bits beside its id
  if (p->max_bounces < 1 || p->max_bounces > (1u << 24) - 1)
    return fail(TPMC_EINVAL, "max_bounces must be in [1, 2^24 - 1]");
  if (p->precision != TPMC_FP32 && p->precision != TPMC_FP64) return fail(TPMC_EINVAL, "unknown precision");
  if (p->cv_kind > TPMC_CV_BOX_MAXWELL) return fail(TPMC_EINVAL, "unknown cv_kind");
  if (!std::isfinite(p->l_ref)) return fail(TPMC_EINVAL, "l_ref must be finite");
  if (p->gsi_model > TPMC_GSI_CLL) return fail(TPMC_EINVAL, "unknown gsi_model");
  if (p->gsi_model == TPMC_GSI_CLL &&
      !(p->alpha_n >= 0.0 && p->alpha_n <= 1.0 && p->sigma_t >= 0.0 && p->sigma_t <= 1.0))
    return fail(TPMC_EINVAL, "CLL: alpha_n and sigma_t must be in [0, 1]");
  if (p->cv_kind != TPMC_CV_SPHERE)
    for (int i = 0; i < 3; ++i)
      if (!(std::isfinite(p->box_lo[i]) && std::isfinite(p->box_hi[i]) && p->box_hi[i] > p->box_lo[i]))
        return fail(TPMC_EINVAL, "box CV: box_lo and box_hi must be finite with box_hi > box_lo");
  return TPMC_OK;
}

tpmc_status fill_query(const MeshRec& m, const tpmc_params* p, uint64_t N, QueryDev* q) {
  std::memset(q, 0, sizeof(*q));
  q->n = p->n; q->T_inf = p->T_inf; q->m = p->m; q->V = p->V;
  for (int i = 0; i < 3; ++i) { q->dir[i] = p->dir[i]; q->ref[i] = p->ref_point[i]; }
  q->T_W = p->T_W; q->eps = p->eps_diffuse; q->A_ref = p->A_ref;
  // The Maxwell choice u < eps on the uniform u = (k + 1/2) 2^-23 of a draw's
  // top 23 bits k holds exactly when k < eps 2^23 - 1/2, i.e. k < ceil(eps 2^23 - 1/2)
  // (eps 2^23 - 1/2 is exact in double), so the kernel decides in integers.
  q->eps_k = (uint32_t)std::min(8388608.0, std::max(0.0, std::ceil(p->eps_diffuse * 8388608.0 - 0.5)));
  q->l_ref = p->l_ref > 0.0 ? p->l_ref : 1.0;
  q->cv_kind = p->cv_kind;
  q->gsi_model = p->gsi_model;
  if (p->gsi_model == TPMC_GSI_CLL) {
    const double at = p->sigma_t * (2.0 - p->sigma_t);
    const double c[4] = {p->alpha_n, std::sqrt(1.0 - p->alpha_n), at, std::sqrt(std::max(0.0, 1.0 - at))};
    for (int i = 0; i < 4; ++i) { q->cll[i] = c[i]; q->fcll[i] = (float)c[i]; }
  }
  if (p->cv_kind != TPMC_CV_SPHERE) {
    // box CV: the body must lie strictly inside the box
    for (int i = 0; i < 3; ++i) {
      q->box_lo[i] = p->box_lo[i];
      q->box_hi[i] = p->box_hi[i];
      q->center[i] = 0.5 * (p->box_lo[i] + p->box_hi[i]);
    }
    q->r_cv = 0.0;
    for (uint64_t k = 0; k < m.h_tri.size(); ++k) {
      const double* v = &m.h_xyz[3 * (size_t)m.h_tri[k]];
      for (int i = 0; i < 3; ++i)
        if (!(v[i] > q->box_lo[i] && v[i] < q->box_hi[i]))
          return fail(TPMC_EINVAL, "the mesh is not strictly inside the box control volume");
    }
  } else if (p->r_cv <= 0.0) {
    for (int i = 0; i < 3; ++i) q->center[i] = m.center[i];
    q->r_cv = m.radius > 0.0 ? 1.05 * m.radius : 1.0;
  } else {
    for (int i = 0; i < 3; ++i) q->center[i] = p->center[i];
    q->r_cv = p->r_cv;
    // the body must lie strictly inside the control volume
    double far2 = 0.0;
    for (uint64_t k = 0; k < m.h_tri.size(); ++k) {
      const double* v = &m.h_xyz[3 * (size_t)m.h_tri[k]];
      double d2 = 0.0;
      for (int i = 0; i < 3; ++i) d2 += (v[i] - q->center[i]) * (v[i] - q->center[i]);
      far2 = std::max(far2, d2);
    }
    if (!(std::sqrt(far2) < q->r_cv)) return fail(TPMC_EINVAL, "the mesh is not strictly inside the control volume");
  }
  double dref = 0.0;
  for (int i = 0; i < 3; ++i) dref += (m.center[i] - q->ref[i]) * (m.center[i] - q->ref[i]);
  q->rmax = std::sqrt(dref) + m.radius;
  q->N = N;
  q->seed = p->seed;
  q->stream_id = p->stream_id;
  q->max_bounces = p->max_bounces;
  q->precision = p->precision;
  q->panel = nullptr;
  return TPMC_OK;
}

LaunchCfg Ctx::schedule(const MeshRec& m, uint32_t variant, uint64_t total) {
  LaunchCfg cfg;
  const uint64_t key = tune_key(m.dev.n_tri, variant);
  auto it = tuned.find(key);
  if (manual_launch) cfg = manual;
  else if (it != tuned.end()) cfg = it->second;
  else {
    // Untuned default, from same-box sweeps on GB300 with the current kernel
    // at 96 cases x 2e6 and x 1e7 particles per launch: 128 threads at the
    // highest occupancy (8 blocks per SM) for every tree.  Against 256 x 2
    // (no register cap) the plate is 4-8 % faster, the cylinder 25 %, the
    // satellite 23 %; against 6 blocks per SM the cylinder 9 % and the
    // satellite 10 % faster, the diffuse plate 0.6 % slower.
    cfg.block = 128;
    cfg.smem_nodes = 0;  // the hot top of the tree stays in L1; shared-memory staging costs bank conflicts
    cfg.blocks_per_sm = 0;
    cfg.chunk = 0;
  }
  cfg.smem_nodes = m.dev.width > 2 ? 0u : std::min<uint32_t>(cfg.smem_nodes, m.dev.n_nodes);  // wide: none staged
  // A traversal round ends once this many lanes have finished their rays.
  // Same-box sweeps with the current kernel: 16 to 28 are equal on the plate
  // and the cylinder; on the satellite 16 is 3 % faster than 24 and 2 % than 20.
  if (cfg.refill_at == 0 || cfg.refill_at > 32) cfg.refill_at = 16;
  const int maxb = trace_max_blocks_per_sm(variant, cfg, m.dev.n_nodes);
  if (cfg.blocks_per_sm == 0 || (int)cfg.blocks_per_sm > maxb) cfg.blocks_per_sm = std::max(1, maxb);
  if (cfg.chunk == 0) {
    const uint64_t warps = (uint64_t)num_sms * cfg.blocks_per_sm * (cfg.block / 32);
    uint64_t ch = total / std::max<uint64_t>(1, warps * 16);
    ch = (ch / 32) * 32;
    cfg.chunk = (uint32_t)std::min<uint64_t>(1024, std::max<uint64_t>(32, ch));
  }
  return cfg;
}

// One batched run: nq queries prepared on the device from `base` (+ dirs/S)
// or uploaded one by one, traced together, finalised into d_out.
tpmc_status Ctx::run(const MeshRec& m, const QueryDev* h_queries, uint32_t nq, const QueryDev* h_base,
                     const double* d_dirs, const double* d_S, const ItemDev* h_items, uint32_t n_items, uint64_t total,
                     uint32_t variant, tpmc_result* d_out, const RecordsDev* rec) {
  tpmc_status st;
  if ((st = grow(s_queries, sizeof(QueryDev) * (size_t)nq, "queries")) != TPMC_OK) return st;
  if ((st = grow(s_acc, sizeof(AccStripe) * kAccStripes * (size_t)nq, "accumulators")) != TPMC_OK) return st;
  if ((st = grow(s_items, sizeof(ItemDev) * (size_t)std::max(nq, n_items), "work items")) != TPMC_OK) return st;
  if ((st = grow(s_misc, 256, "counters")) != TPMC_OK) return st;
  if ((st = grow(s_base, sizeof(QueryDev), "base query")) != TPMC_OK) return st;
  QueryDev* d_queries = (QueryDev*)s_queries.ptr;
  AccStripe* d_acc = (AccStripe*)s_acc.ptr;
  ItemDev* d_items = (ItemDev*)s_items.ptr;
  unsigned long long* d_counter = (unsigned long long*)s_misc.ptr;
  int* d_err = (int*)((char*)s_misc.ptr + 64);
  cudaError_t e;
  // Host sources here are pageable, so each copy is staged before the call
  // returns and the caller's structs may be reused at once.
  if (h_base) {
    if ((e = cudaMemcpyAsync(s_base.ptr, h_base, sizeof(QueryDev), cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_fail(e, "upload base query");
  } else {
    if ((e = cudaMemcpyAsync(d_queries, h_queries, sizeof(QueryDev) * nq, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_fail(e, "upload queries");
    if ((e = cudaMemcpyAsync(d_items, h_items, sizeof(ItemDev) * n_items, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return cuda_fail(e, "upload items");
  }
  if ((e = cudaMemsetAsync(s_misc.ptr, 0, 128, stream)) != cudaSuccess) return cuda_fail(e, "clear counter");
  // the set-up also clears the queries' accumulators
  if ((e = launch_setup(d_queries, nq, h_base ? (const QueryDev*)s_base.ptr : nullptr, d_dirs, d_S,
                        h_base ? d_items : nullptr, nullptr, d_acc, nq, stream)) != cudaSuccess)
    return cuda_fail(e, "setup kernel");
  TraceArgs a{};
  a.mesh = m.dev;
  a.queries = d_queries;
  a.acc = d_acc;
  a.acc_stride = nq;
  a.items = d_items;
  a.n_items = h_base ? nq : n_items;
  a.total = total;
  a.counter = d_counter;
  a.error = d_err;
  a.count_work = counters ? 1u : 0u;
  a.vn_table = vn_table;
  if (rec) a.rec = *rec;
  const LaunchCfg cfg = schedule(m, variant, total);
  a.chunk = cfg.chunk;
  a.smem_nodes = cfg.smem_nodes;
  a.refill_at = cfg.refill_at;
  last_cfg = cfg;
  if (total > 0 && (e = launch_trace(a, variant, cfg, num_sms, stream)) != cudaSuccess) return cuda_fail(e, "trace kernel");
  if ((e = launch_finalize(d_queries, d_acc, nq, nq, nullptr, d_out, stream)) != cudaSuccess)
    return cuda_fail(e, "finalize kernel");
  if ((e = cudaMemcpyAsync(h_err_word, d_err, sizeof(int), cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return cuda_fail(e, "read error word");
  return TPMC_OK;
}

tpmc_status Ctx::check_error_word() {
  if (*h_err_word != 0) {
    const int w = *h_err_word;
    *h_err_word = 0;
    return fail(TPMC_ECUDA, "trace kernel reported error word " + std::to_string(w) + " (traversal stack overflow)");
  }
  return TPMC_OK;
}

// BVH width of a mesh load: the one set by tpmc_set_launch, else the one
// tpmc_tune chose for the size class, else the default.
uint32_t Ctx::width_for(uint32_t n_tri) const {
  if (bvh_width) return bvh_width;
  auto it = tuned_width.find(tune_key(n_tri, 0));
  return it != tuned_width.end() ? it->second : kDefaultBvhWidth;
}

// Builds the mesh's BVH with `width` children per node and uploads it, its
// triangles and frames into one device allocation (the host copies of the
// mesh are not set here).
tpmc_status Ctx::upload_mesh(const double* xyz, uint32_t n_vert, const uint32_t* tri, uint32_t n_tri, uint32_t width,
                             MeshRec* out) {
  BvhBuild b;
  const char* err = nullptr;
  if (!build_bvh(xyz, n_vert, tri, n_tri, bvh_leaf, width, &b, &err)) {
    b.release();
    return fail(TPMC_EINVAL, err);
  }
  MeshRec& m = *out;
  const size_t sz_nodes = b.n_nodes * b.node_bytes;
  const size_t sz_tris = (size_t)b.n_leaf_tris * 12 * sizeof(float);
  const size_t sz_tris64 = (size_t)b.n_leaf_tris * 12 * sizeof(double);
  const size_t sz_fr = (size_t)n_tri * 8 * sizeof(float);
  const size_t sz_fr64 = (size_t)n_tri * 8 * sizeof(double);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t total = al(sz_nodes) + al(sz_tris) + al(sz_tris64) + al(sz_fr) + al(sz_fr64);
  tpmc_status st = alloc(&m.d_block, std::max(total, (size_t)256), "mesh");
  if (st != TPMC_OK) { b.release(); return st; }
  char* base = (char*)m.d_block;
  size_t off = 0;
  auto place = [&](size_t sz) { char* p = base + off; off += al(sz); return p; };
  char* p_nodes = place(sz_nodes);
  char* p_tris = place(sz_tris);
  char* p_tris64 = place(sz_tris64);
  char* p_fr = place(sz_fr);
  char* p_fr64 = place(sz_fr64);
  cudaError_t e = cudaSuccess;
  if (sz_nodes) e = cudaMemcpy(p_nodes, b.nodes, sz_nodes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && sz_tris) e = cudaMemcpy(p_tris, b.tris, sz_tris, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && sz_tris64) e = cudaMemcpy(p_tris64, b.tris64, sz_tris64, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && sz_fr) e = cudaMemcpy(p_fr, b.frames, sz_fr, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && sz_fr64) e = cudaMemcpy(p_fr64, b.frames64, sz_fr64, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    release(m.d_block);
    m.d_block = nullptr;
    b.release();
    return cuda_fail(e, "upload mesh");
  }
  m.dev.nodes = (const float4*)p_nodes;
  m.dev.tris = (const float4*)p_tris;
  m.dev.tris64 = (const double*)p_tris64;
  m.dev.frames = (const float4*)p_fr;
  m.dev.frames64 = (const double*)p_fr64;
  m.dev.n_nodes = (uint32_t)b.n_nodes;
  m.dev.width = b.width;
  m.dev.depth = b.depth;
  for (int k = 0; k < 3; ++k) {
    // the padded root box (empty when there is no mesh): binary trees test it
    // in their grid's units, wide trees in metres
    m.dev.box_lo[k] = b.width == 2 ? b.qroot_lo[k] : b.root_lo[k];
    m.dev.box_hi[k] = b.width == 2 ? b.qroot_hi[k] : b.root_hi[k];
    m.dev.qorigin[k] = b.qorigin[k];
    m.dev.qstep[k] = b.qstep[k];
  }
  m.dev.n_tri = n_tri;
  m.dev.n_tri_leaf = b.n_leaf_tris;
  m.dev.scene_radius = (float)b.radius;
  for (int i = 0; i < 3; ++i) m.center[i] = b.center[i];
  m.radius = b.radius;
  m.depth = b.depth;
  m.leaf_max = b.leaf_max;
  m.n_skipped = b.n_skipped;
  m.n_exposed = b.n_exposed;
  m.node_bytes = b.node_bytes;
  m.n_vert = n_vert;
  m.bytes = total;
  b.release();
  return TPMC_OK;
}

Ctx::~Ctx() {
  if (serve) stop_serving(this);
  for (auto& kv : panels) release(kv.second.d_panel);
  for (auto& kv : meshes) release(kv.second.d_block);
  for (Scratch* s : {&s_queries, &s_acc, &s_items, &s_misc, &s_base, &s_out, &s_in})
    release(s->ptr);
  release(vn_table);
  if (h_pinned) cudaFreeHost(h_pinned);
  if (own_stream) cudaStreamDestroy(own_stream);
}

}  // namespace tpmc

using namespace tpmc;

// =========================================================================
extern "C" {

tpmc_status tpmc_create(int device, size_t mem_budget_bytes, tpmc_ctx** out) {
  if (!out) return fail(TPMC_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= n) return fail(TPMC_EINVAL, "no such CUDA device");
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  std::unique_ptr<Ctx> c(new Ctx());
  c->device = device;
  cudaDeviceProp prop;
  if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  c->num_sms = prop.multiProcessorCount;
  size_t free_b = 0, total_b = 0;
  if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
  c->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)(0.9 * (double)free_b);
  if ((e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  c->stream = c->own_stream;
  if ((e = cudaMallocHost(&c->h_pinned, 4096)) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
  {
    void* t = nullptr;
    tpmc_status st = c->alloc(&t, sizeof(float) * kVnNS * kVnNZ, "normal-speed table");
    if (st != TPMC_OK) return st;
    c->vn_table = (float*)t;
    if ((e = launch_vn_table(c->vn_table, c->stream)) != cudaSuccess) return cuda_fail(e, "normal-speed table");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(e, "normal-speed table");
  }
  c->h_err_word = (int*)c->h_pinned;
  *c->h_err_word = 0;
  *out = reinterpret_cast<tpmc_ctx*>(c.release());
  return TPMC_OK;
}

tpmc_status tpmc_destroy(tpmc_ctx* ctx) {
  if (!ctx) return TPMC_OK;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  delete c;
  return TPMC_OK;
}

tpmc_status tpmc_set_stream(tpmc_ctx* ctx, void* cuda_stream) {
  if (!ctx) return fail(TPMC_EINVAL, "ctx is NULL");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  c->stream = cuda_stream ? (cudaStream_t)cuda_stream : c->own_stream;
  return TPMC_OK;
}

const char* tpmc_last_error(const tpmc_ctx*) { return g_last_error.c_str(); }

tpmc_status tpmc_memory_info(tpmc_ctx* ctx, size_t* used, size_t* budget, uint64_t* n_allocs) {
  if (!ctx) return fail(TPMC_EINVAL, "ctx is NULL");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  if (used) *used = c->used;
  if (budget) *budget = c->budget;
  if (n_allocs) *n_allocs = c->n_allocs;
  return TPMC_OK;
}

tpmc_status tpmc_set_counters(tpmc_ctx* ctx, int enable) {
  if (!ctx) return fail(TPMC_EINVAL, "ctx is NULL");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  c->counters = enable != 0;
  return TPMC_OK;
}

tpmc_status tpmc_mesh_load(tpmc_ctx* ctx, const double* xyz, uint32_t n_vert, const uint32_t* tri, uint32_t n_tri,
                           tpmc_mesh_id* out) {
  if (!ctx || !out) return fail(TPMC_EINVAL, "NULL argument");
  if ((n_vert > 0 && !xyz) || (n_tri > 0 && !tri)) return fail(TPMC_EINVAL, "NULL mesh array");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  MeshRec m;
  tpmc_status st = c->upload_mesh(xyz, n_vert, tri, n_tri, c->width_for(n_tri), &m);
  if (st != TPMC_OK) return st;
  m.h_xyz.assign(xyz, xyz + 3 * (size_t)n_vert);
  m.h_tri.assign(tri, tri + 3 * (size_t)n_tri);
  const tpmc_mesh_id id = c->next_mesh++;
  c->meshes[id] = std::move(m);
  *out = id;
  return TPMC_OK;
}

tpmc_status tpmc_mesh_unload(tpmc_ctx* ctx, tpmc_mesh_id mesh) {
  if (!ctx) return fail(TPMC_EINVAL, "ctx is NULL");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  auto it = c->meshes.find(mesh);
  if (it == c->meshes.end()) return fail(TPMC_ENOTFOUND, "unknown mesh id");
  if (it->second.in_use > 0) return fail(TPMC_EBUSY, "mesh is used by queries in flight");
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  c->release(it->second.d_block);
  c->meshes.erase(it);
  return TPMC_OK;
}

tpmc_status tpmc_mesh_info(tpmc_ctx* ctx, tpmc_mesh_id mesh, tpmc_mesh_stats* out) {
  if (!ctx || !out) return fail(TPMC_EINVAL, "NULL argument");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  auto it = c->meshes.find(mesh);
  if (it == c->meshes.end()) return fail(TPMC_ENOTFOUND, "unknown mesh id");
  const MeshRec& m = it->second;
  std::memset(out, 0, sizeof(*out));
  out->n_tri = m.dev.n_tri;
  out->n_vert = m.n_vert;
  out->n_nodes = m.dev.n_nodes;
  out->depth = m.depth;
  out->n_skipped = m.n_skipped;
  out->leaf_max = m.leaf_max;
  for (int i = 0; i < 3; ++i) out->bound_center[i] = m.center[i];
  out->bound_radius = m.radius;
  out->device_bytes = m.bytes;
  out->n_refs = m.dev.n_tri_leaf;
  out->n_exposed = m.n_exposed;
  out->bvh_width = m.dev.width;
  out->node_bytes = m.node_bytes;
  return TPMC_OK;
}

static tpmc_status trace_common(Ctx* c, tpmc_mesh_id mesh, const tpmc_params* params, uint64_t N,
                                tpmc_records* records, tpmc_result* out) {
  if (!out) return fail(TPMC_EINVAL, "out is NULL");
  tpmc_status st = validate_params(params);
  if (st != TPMC_OK) return st;
  if (N == 0 || N > (1ull << 34)) return fail(TPMC_EINVAL, "N must be in [1, 2^34]");
  auto it = c->meshes.find(mesh);
  if (it == c->meshes.end()) return fail(TPMC_ENOTFOUND, "unknown mesh id");
  const MeshRec& m = it->second;
  cudaSetDevice(c->device);
  const auto t0 = std::chrono::steady_clock::now();
  QueryDev q;
  if ((st = fill_query(m, params, N, &q)) != TPMC_OK) return st;
  // per-triangle loads
  void* d_panel = nullptr;
  if (params->want_panels && m.dev.n_tri > 0) {
    if ((st = c->alloc(&d_panel, (size_t)m.dev.n_tri * 3 * sizeof(long long), "panel loads")) != TPMC_OK) return st;
    cudaMemsetAsync(d_panel, 0, (size_t)m.dev.n_tri * 3 * sizeof(long long), c->stream);
    q.panel = (long long*)d_panel;
  }
  // records
  RecordsDev rec;
  void* d_rec = nullptr;
  if (records) {
    if (records->K > (uint32_t)kMaxRecordK || N > (1ull << 26)) {
      c->release(d_panel);
      return fail(TPMC_EINVAL, "records: K must be <= 64 and N <= 2^26");
    }
    const size_t K = std::max<uint32_t>(records->K, 1);
    const size_t bytes = N * (9 * sizeof(double) + (2 + K) * sizeof(uint32_t));
    if ((st = c->alloc(&d_rec, bytes, "records")) != TPMC_OK) { c->release(d_panel); return st; }
    char* p = (char*)d_rec;
    rec.pos = (double*)p; p += N * 3 * sizeof(double);
    rec.vel = (double*)p; p += N * 3 * sizeof(double);
    rec.dv = (double*)p; p += N * 3 * sizeof(double);
    rec.n_hits = (uint32_t*)p; p += N * sizeof(uint32_t);
    rec.truncated = (uint32_t*)p; p += N * sizeof(uint32_t);
    rec.tri = (uint32_t*)p;
    rec.K = records->K;
    cudaMemsetAsync(rec.tri, 0xFF, N * K * sizeof(uint32_t), c->stream);
  }
  ItemDev item;
  std::memset(&item, 0, sizeof(item));
  item.g_begin = 0; item.pid_begin = 0; item.count = N; item.query = 0;
  tpmc_status rs = c->grow(c->s_out, sizeof(tpmc_result), "result");
  if (rs == TPMC_OK)
    rs = c->run(m, &q, 1, nullptr, nullptr, nullptr, &item, 1, N, trace_variant(params, m.dev), (tpmc_result*)c->s_out.ptr,
                records ? &rec : nullptr);
  cudaError_t e = cudaSuccess;
  if (rs == TPMC_OK) e = cudaMemcpyAsync(out, c->s_out.ptr, sizeof(tpmc_result), cudaMemcpyDeviceToHost, c->stream);
  if (rs == TPMC_OK && e == cudaSuccess && records) {
    const size_t K = records->K;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
      if (dst && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
    };
    cp(records->pos, rec.pos, N * 3 * sizeof(double));
    cp(records->vel, rec.vel, N * 3 * sizeof(double));
    cp(records->dv, rec.dv, N * 3 * sizeof(double));
    cp(records->n_hits, rec.n_hits, N * sizeof(uint32_t));
    cp(records->truncated, rec.truncated, N * sizeof(uint32_t));
    if (K) cp(records->tri, rec.tri, N * K * sizeof(uint32_t));
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (d_rec) c->release(d_rec);
  if (rs != TPMC_OK || e != cudaSuccess) {
    c->release(d_panel);
    return rs != TPMC_OK ? rs : cuda_fail(e, "trace");
  }
  if ((st = c->check_error_word()) != TPMC_OK) { c->release(d_panel); return st; }
  const auto t1 = std::chrono::steady_clock::now();
  out->ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  if (out->status != TPMC_OK) {
    c->release(d_panel);
    return fail((tpmc_status)out->status, "query set-up rejected the parameters (S outside [0.01, 50] or fixed-point range)");
  }
  out->query_id = c->next_query++;
  if (d_panel) {
    PanelRec pr;
    pr.d_panel = d_panel;
    pr.query = q;
    pr.mesh = mesh;
    pr.n_tri = m.dev.n_tri;
    // keep the set-up values the panel conversion needs
    pr.query.gamma = out->gamma;
    pr.query.m = params->m;
    pr.query.c_mp = out->c_mp;
    pr.query.quantum = out->fixed_quantum;
    c->panels[out->query_id] = pr;
  }
  return TPMC_OK;
}

tpmc_status tpmc_trace(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* params, uint64_t N, tpmc_result* out) {
  if (!ctx) return fail(TPMC_EINVAL, "ctx is NULL");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  return trace_common(c, mesh, params, N, nullptr, out);
}

tpmc_status tpmc_trace_records(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* params, uint64_t N,
                               tpmc_records* records, tpmc_result* out) {
  if (!ctx || !records) return fail(TPMC_EINVAL, "NULL argument");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  return trace_common(c, mesh, params, N, records, out);
}

static tpmc_status panels_locked(Ctx* c, tpmc_query_id query, double* pressure, double* shear, uint32_t n_tri) {
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  auto it = c->panels.find(query);
  if (it == c->panels.end()) return fail(TPMC_ENOTFOUND, "no panel loads kept for this query");
  PanelRec& pr = it->second;
  if (n_tri != pr.n_tri) return fail(TPMC_EINVAL, "n_tri does not match the mesh");
  auto mit = c->meshes.find(pr.mesh);
  if (mit == c->meshes.end()) return fail(TPMC_ENOTFOUND, "the query's mesh was unloaded");
  cudaSetDevice(c->device);
  tpmc_status st;
  if ((st = c->grow(c->s_in, sizeof(QueryDev), "panel query")) != TPMC_OK) return st;
  void* d_pv = nullptr;
  if ((st = c->alloc(&d_pv, (size_t)n_tri * 2 * sizeof(double), "panel output")) != TPMC_OK) return st;
  double* d_p = (double*)d_pv;
  double* d_s = d_p + n_tri;
  cudaError_t e = cudaMemcpyAsync(c->s_in.ptr, &pr.query, sizeof(QueryDev), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = launch_panels((const QueryDev*)c->s_in.ptr, (const long long*)pr.d_panel, mit->second.dev.frames,
                      mit->second.dev.frames64, n_tri, d_p, d_s, c->stream);
  if (e == cudaSuccess && pressure) e = cudaMemcpyAsync(pressure, d_p, n_tri * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && shear) e = cudaMemcpyAsync(shear, d_s, n_tri * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  c->release(d_pv);
  if (e != cudaSuccess) return cuda_fail(e, "panels");
  c->release(pr.d_panel);
  c->panels.erase(it);
  return TPMC_OK;
}

tpmc_status tpmc_panels(tpmc_ctx* ctx, tpmc_query_id query, double* pressure, double* shear, uint32_t n_tri) {
  if (!ctx) return fail(TPMC_EINVAL, "ctx is NULL");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  const tpmc_status st = panels_locked(c, query, pressure, shear, n_tri);
  // after the context lock is dropped (the scheduler takes its own lock first)
  if (st == TPMC_OK) serve_memory_released(c);
  return st;
}

tpmc_status tpmc_panel_sums(tpmc_ctx* ctx, tpmc_query_id query, int64_t* dv_q, uint32_t n_tri) {
  if (!ctx) return fail(TPMC_EINVAL, "ctx is NULL");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!dv_q) return fail(TPMC_EINVAL, "dv_q is NULL");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  auto it = c->panels.find(query);
  if (it == c->panels.end()) return fail(TPMC_ENOTFOUND, "no panel loads kept for this query");
  const PanelRec& pr = it->second;
  if (n_tri != pr.n_tri) return fail(TPMC_EINVAL, "n_tri does not match the mesh");
  cudaSetDevice(c->device);
  cudaError_t e = cudaMemcpyAsync(dv_q, pr.d_panel, (size_t)n_tri * 3 * sizeof(long long), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "panel sums");
  return TPMC_OK;
}

static tpmc_status sweep_common(Ctx* c, tpmc_mesh_id mesh, const tpmc_params* base, const double* d_dirs,
                                const double* d_S, uint32_t K, uint64_t N_each, tpmc_result* d_out) {
  tpmc_status st = validate_params(base);
  if (st != TPMC_OK) return st;
  if (K == 0 || K > kMaxLaunchQueries) return fail(TPMC_EINVAL, "K must be in [1, 2^24]");
  if (N_each == 0 || N_each > (1ull << 34)) return fail(TPMC_EINVAL, "N_each must be in [1, 2^34]");
  if ((uint64_t)K * N_each > (1ull << 50)) return fail(TPMC_EINVAL, "K * N_each too large");
  auto it = c->meshes.find(mesh);
  if (it == c->meshes.end()) return fail(TPMC_ENOTFOUND, "unknown mesh id");
  const MeshRec& m = it->second;
  QueryDev q;
  if ((st = fill_query(m, base, N_each, &q)) != TPMC_OK) return st;
  return c->run(m, nullptr, K, &q, d_dirs, d_S, nullptr, 0, (uint64_t)K * N_each, trace_variant(base, m.dev), d_out, nullptr);
}

tpmc_status tpmc_sweep(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* base, const double* h_dirs,
                       const double* h_S, uint32_t K, uint64_t N_each, tpmc_result* h_out) {
  if (!ctx || !h_out) return fail(TPMC_EINVAL, "NULL argument");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  const auto t0 = std::chrono::steady_clock::now();
  tpmc_status st;
  const size_t in_bytes = (size_t)K * 4 * sizeof(double);
  if ((st = c->grow(c->s_in, std::max(in_bytes, sizeof(QueryDev)), "sweep inputs")) != TPMC_OK) return st;
  if ((st = c->grow(c->s_out, (size_t)K * sizeof(tpmc_result), "sweep results")) != TPMC_OK) return st;
  double* d_dirs = h_dirs ? (double*)c->s_in.ptr : nullptr;
  double* d_S = h_S ? (double*)c->s_in.ptr + 3 * (size_t)K : nullptr;
  cudaError_t e = cudaSuccess;
  if (h_dirs) e = cudaMemcpyAsync(d_dirs, h_dirs, (size_t)K * 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && h_S) e = cudaMemcpyAsync(d_S, h_S, (size_t)K * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "upload sweep inputs");
  if ((st = sweep_common(c, mesh, base, d_dirs, d_S, K, N_each, (tpmc_result*)c->s_out.ptr)) != TPMC_OK) return st;
  e = cudaMemcpyAsync(h_out, c->s_out.ptr, (size_t)K * sizeof(tpmc_result), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sweep");
  if ((st = c->check_error_word()) != TPMC_OK) return st;
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (uint32_t k = 0; k < K; ++k) h_out[k].ms = ms;
  return TPMC_OK;
}

tpmc_status tpmc_sweep_device(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* base, const double* d_dirs,
                              const double* d_S, uint32_t K, uint64_t N_each, tpmc_result* d_out) {
  if (!ctx || !d_out) return fail(TPMC_EINVAL, "NULL argument");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return sweep_common(c, mesh, base, d_dirs, d_S, K, N_each, d_out);
}

tpmc_status tpmc_set_launch(tpmc_ctx* ctx, const tpmc_launch* cfg) {
  if (!ctx) return fail(TPMC_EINVAL, "ctx is NULL");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  if (!cfg) {
    c->manual_launch = false;
    c->bvh_leaf = 4;
    c->bvh_width = 0;
    return TPMC_OK;
  }
  if (cfg->bvh_leaf > 127) return fail(TPMC_EINVAL, "bvh_leaf must be in [0, 127]");
  if (cfg->bvh_width != 0 && cfg->bvh_width != 2 && cfg->bvh_width != 4 && cfg->bvh_width != 8)
    return fail(TPMC_EINVAL, "bvh_width must be 0, 2, 4 or 8");
  if (cfg->block == 0) {  // the BVH layout of later loads only
    c->bvh_leaf = cfg->bvh_leaf ? cfg->bvh_leaf : 4;
    c->bvh_width = cfg->bvh_width;
    return TPMC_OK;
  }
  if (cfg->block % 32 != 0 || cfg->block > 256) return fail(TPMC_EINVAL, "block must be 32..256, multiple of 32");
  if (cfg->chunk != 0 && (cfg->chunk % 32 != 0)) return fail(TPMC_EINVAL, "chunk must be a multiple of 32");
  if (cfg->refill_at > 32) return fail(TPMC_EINVAL, "refill_at must be in [0, 32]");
  if (cfg->bvh_leaf > 127) return fail(TPMC_EINVAL, "bvh_leaf must be in [0, 127]");
  c->manual_launch = true;
  c->manual.block = cfg->block;
  c->manual.blocks_per_sm = cfg->blocks_per_sm;
  c->manual.chunk = cfg->chunk;
  c->manual.smem_nodes = cfg->smem_nodes;
  c->manual.refill_at = cfg->refill_at;
  c->bvh_leaf = cfg->bvh_leaf ? cfg->bvh_leaf : 4;
  c->bvh_width = cfg->bvh_width;
  return TPMC_OK;
}

tpmc_status tpmc_get_launch(tpmc_ctx* ctx, tpmc_mesh_id mesh, uint32_t precision, tpmc_launch* out) {
  if (!ctx || !out) return fail(TPMC_EINVAL, "NULL argument");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  auto it = c->meshes.find(mesh);
  if (it == c->meshes.end()) return fail(TPMC_ENOTFOUND, "unknown mesh id");
  const LaunchCfg cfg = c->schedule(
      it->second, precision | (it->second.dev.width == 8 ? kVariantWide8 : (it->second.dev.width == 4 ? kVariantWide4 : 0u)), 0);
  out->block = cfg.block;
  out->blocks_per_sm = cfg.blocks_per_sm;
  out->chunk = cfg.chunk;
  out->smem_nodes = cfg.smem_nodes;
  out->refill_at = cfg.refill_at;
  out->bvh_leaf = c->bvh_leaf;
  out->bvh_width = it->second.dev.width;
  return TPMC_OK;
}

}  // extern "C"
