// Autotuner of the trace kernel: BVH layout and launch schedule.
//
// Three stages, each timed with CUDA events on runs of the caller's query:
//   1. BVH width: the mesh is laid out with 2, 4 and 8 children per node (from
//      the context's host copy of it) and each layout runs the untuned
//      schedule; the fastest layout replaces the mesh's own (unless queries
//      in flight use the mesh) and becomes the width of later loads of
//      meshes of its size class;
//   2. schedule on that layout: threads per block, resident blocks per SM (the
//      highest occupancy, 6 and 4), the traversal-round refill threshold and
//      the BVH nodes staged in shared memory (0, 64, 256, 1024);
//   3. particles per lane: the work a warp takes per fetch from the global
//      counter, 32 x {1, 2, 4, 8, 16, 32} ids, against the automatic size.
// The schedule is kept for the mesh's size class (powers of 4 of the triangle
// count) and kernel variant; later launches on meshes of that class use it.
#include <algorithm>
#include <cstring>
#include <vector>

#include "runtime.h"

using namespace tpmc;

namespace {

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Timer() {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  ~Timer() {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
};

// Marginal rate (particles per ms) of schedule `cfg` on mesh `m`: the query
// traces N_trial / 4 and then N_trial particles, and the rate is the
// difference in particles over the difference in time, so that the fixed
// costs of a launch (set-up, reduction, the tail of its last warps) drop out
// and the choice holds for the long launches of sweeps.  `used` receives the
// schedule as completed by Ctx::schedule.
tpmc_status measure(Ctx* c, const MeshRec& m, const tpmc_params* params, uint64_t N_trial, const LaunchCfg& cfg,
                    bool manual, Timer& tm, double* rate, LaunchCfg* used) {
  QueryDev q;
  tpmc_status st = fill_query(m, params, N_trial, &q);
  if (st != TPMC_OK) return st;
  ItemDev item;
  std::memset(&item, 0, sizeof(item));
  const bool had_manual = c->manual_launch;
  const LaunchCfg old_manual = c->manual;
  c->manual_launch = manual;
  c->manual = cfg;
  const uint64_t quarter = std::max<uint64_t>(1, N_trial / 4);
  float ms[2] = {0.0f, 0.0f};
  for (int k = 0; k < 2 && st == TPMC_OK; ++k) {
    item.count = k == 0 ? quarter : N_trial;
    q.N = item.count;
    cudaEventRecord(tm.e0, c->stream);
    st = c->run(m, &q, 1, nullptr, nullptr, nullptr, &item, 1, item.count, trace_variant(params, m.dev),
                (tpmc_result*)c->s_out.ptr, nullptr);
    cudaEventRecord(tm.e1, c->stream);
    if (st != TPMC_OK) break;
    const cudaError_t e = cudaEventSynchronize(tm.e1);
    if (e != cudaSuccess) { st = cuda_fail(e, "tune"); break; }
    cudaEventElapsedTime(&ms[k], tm.e0, tm.e1);
    if (used) *used = c->last_cfg;
  }
  c->manual_launch = had_manual;
  c->manual = old_manual;
  if (st != TPMC_OK) return st;
  if ((st = c->check_error_word()) != TPMC_OK) return st;
  const double dt = (double)ms[1] - (double)ms[0];
  *rate = (N_trial > quarter && dt > 0.0) ? (double)(N_trial - quarter) / dt
                                          : (double)N_trial / std::max((double)ms[1], 1e-6);
  return TPMC_OK;
}

// Best of two passes (the first also warms caches and clocks).
tpmc_status measure2(Ctx* c, const MeshRec& m, const tpmc_params* params, uint64_t N_trial, const LaunchCfg& cfg,
                     bool manual, Timer& tm, double* rate, LaunchCfg* used) {
  double r0 = 0.0, r1 = 0.0;
  tpmc_status st = measure(c, m, params, N_trial, cfg, manual, tm, &r0, used);
  if (st == TPMC_OK) st = measure(c, m, params, N_trial, cfg, manual, tm, &r1, used);
  *rate = std::max(r0, r1);
  return st;
}

}  // namespace

extern "C" tpmc_status tpmc_tune(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* params, uint64_t N_trial,
                                 tpmc_launch* best) {
  if (!ctx) return fail(TPMC_EINVAL, "ctx is NULL");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  tpmc_status st = validate_params(params);
  if (st != TPMC_OK) return st;
  if (N_trial == 0 || N_trial > (1ull << 30)) return fail(TPMC_EINVAL, "N_trial must be in [1, 2^30]");
  auto it = c->meshes.find(mesh);
  if (it == c->meshes.end()) return fail(TPMC_ENOTFOUND, "unknown mesh id");
  MeshRec& m = it->second;
  cudaSetDevice(c->device);
  {
    QueryDev q;
    if ((st = fill_query(m, params, N_trial, &q)) != TPMC_OK) return st;
  }
  if ((st = c->grow(c->s_out, sizeof(tpmc_result), "result")) != TPMC_OK) return st;
  Timer tm;
  const uint32_t n_tri = m.dev.n_tri;

  // 1. BVH width, each layout with its untuned schedule
  uint32_t best_width = m.dev.width;
  {
    double best_rate = -1.0;
    MeshRec best_rec;
    bool best_is_new = false;
    const bool may_replace = m.in_use == 0;
    for (uint32_t w : {2u, 4u, 8u}) {
      if (w != m.dev.width && !may_replace) continue;
      MeshRec cand;
      const MeshRec* run_on = &m;
      if (w != m.dev.width) {
        if (c->upload_mesh(m.h_xyz.data(), m.n_vert, m.h_tri.data(), n_tri, w, &cand) != TPMC_OK) continue;
        if (cand.dev.width != w) {  // too deep for the wide stack: kept binary
          c->release(cand.d_block);
          continue;
        }
        run_on = &cand;
      }
      double rate = 0.0;
      st = measure2(c, *run_on, params, N_trial, LaunchCfg(), false, tm, &rate, nullptr);
      if (st != TPMC_OK) {
        if (run_on == &cand) c->release(cand.d_block);
        return st;
      }
      if (rate > best_rate) {
        best_rate = rate;
        best_width = w;
        if (best_is_new) c->release(best_rec.d_block);
        best_is_new = run_on == &cand;
        if (best_is_new) best_rec = cand;
      } else if (run_on == &cand) {
        c->release(cand.d_block);
      }
    }
    if (best_is_new) {
      // the fastest layout replaces the mesh's own (no query uses the mesh)
      cudaStreamSynchronize(c->stream);
      c->release(m.d_block);
      best_rec.h_xyz.swap(m.h_xyz);
      best_rec.h_tri.swap(m.h_tri);
      best_rec.in_use = m.in_use;
      m = std::move(best_rec);
    }
    c->tuned_width[tune_key(n_tri, 0)] = best_width;
  }
  const uint32_t variant = trace_variant(params, m.dev);

  // 2. schedule on the chosen layout
  std::vector<LaunchCfg> cands;
  const uint32_t nn = m.dev.n_nodes;
  for (uint32_t block : {64u, 128u, 256u})
    for (uint32_t sm_nodes : {0u, 64u, 256u, 1024u}) {
      if (sm_nodes > 0 && sm_nodes >= 2 * nn && sm_nodes != 64u) continue;  // a larger stage of a small tree adds nothing
      if (sm_nodes > 0 && m.dev.width > 2) continue;  // only the binary traversal stages nodes
      for (uint32_t occ : {0u, 6u, 4u})  // 0: the highest occupancy
        for (uint32_t refill : {8u, 16u, 24u}) {
          LaunchCfg cfg;
          cfg.block = block;
          cfg.smem_nodes = std::min(sm_nodes, nn);
          cfg.refill_at = refill;
          const int maxb = trace_max_blocks_per_sm(variant, cfg, nn);
          if (maxb < 1 || (occ != 0 && occ >= (uint32_t)maxb)) continue;
          cfg.blocks_per_sm = occ == 0 ? (uint32_t)maxb : occ;
          cfg.chunk = 0;
          cands.push_back(cfg);
        }
    }
  double best_rate = -1.0;
  LaunchCfg best_cfg;
  for (const LaunchCfg& cfg : cands) {
    double rate = 0.0;
    LaunchCfg used;
    if ((st = measure2(c, m, params, N_trial, cfg, true, tm, &rate, &used)) != TPMC_OK) return st;
    if (rate > best_rate) {
      best_rate = rate;
      best_cfg = used;
      best_cfg.chunk = 0;
    }
  }

  // 3. particles per lane: a fixed chunk of 32 k ids per warp fetch, or automatic
  for (uint32_t per_lane : {1u, 2u, 4u, 8u, 16u, 32u}) {
    LaunchCfg cfg = best_cfg;
    cfg.chunk = 32u * per_lane;
    double rate = 0.0;
    LaunchCfg used;
    if ((st = measure2(c, m, params, N_trial, cfg, true, tm, &rate, &used)) != TPMC_OK) return st;
    if (rate > best_rate * 1.005) {  // a fixed chunk must beat the automatic one by more than the noise
      best_rate = rate;
      best_cfg = used;
    }
  }

  c->tuned[tune_key(n_tri, variant)] = best_cfg;
  if (best) {
    best->block = best_cfg.block;
    best->blocks_per_sm = best_cfg.blocks_per_sm;
    best->chunk = best_cfg.chunk;
    best->smem_nodes = best_cfg.smem_nodes;
    best->refill_at = best_cfg.refill_at;
    best->bvh_leaf = c->bvh_leaf;
    best->bvh_width = best_width;
  }
  return TPMC_OK;
}
