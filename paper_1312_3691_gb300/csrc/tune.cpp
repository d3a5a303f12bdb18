// Autotuner of the trace kernel: BVH layout and launch schedule.
//
// Three stages, each timed with CUDA events on a trial sweep of the caller's
// query over eight flow directions (its own, the six axes and a diagonal):
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

// Flow directions of the trial sweep: the caller's and seven fixed ones (the
// axes and a diagonal), so that a schedule is judged on attitudes around the
// whole body, as sweeps and served queries see it.
constexpr int kTrialDirs = 8;
void trial_dirs(const tpmc_params* p, double out[kTrialDirs * 3]) {
  const double fixed[7][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
                              {0.57735026918962576, 0.57735026918962576, 0.57735026918962576}};
  for (int i = 0; i < 3; ++i) out[i] = p->dir[i];
  for (int k = 0; k < 7; ++k)
    for (int i = 0; i < 3; ++i) out[3 * (k + 1) + i] = fixed[k][i];
}

// Marginal rate (particles per ms) of schedule `cfg` on mesh `m`: a sweep of
// the kTrialDirs directions traces N_trial / 4 and then N_trial particles in
// all, and the rate is the difference in particles over the difference in
// time, so that the fixed costs of a launch (set-up, reduction, the tail of
// its last warps) drop out and the choice holds for the long launches of
// sweeps.  `used` receives the schedule as completed by Ctx::schedule.
tpmc_status measure(Ctx* c, const MeshRec& m, const tpmc_params* params, uint64_t N_trial, const double* d_dirs,
                    const LaunchCfg& cfg, bool manual, Timer& tm, double* rate, LaunchCfg* used) {
  const bool had_manual = c->manual_launch;
  const LaunchCfg old_manual = c->manual;
  c->manual_launch = manual;
  c->manual = cfg;
  const uint64_t each[2] = {std::max<uint64_t>(1, N_trial / (4 * kTrialDirs)), std::max<uint64_t>(1, N_trial / kTrialDirs)};
  float ms[2] = {0.0f, 0.0f};
  tpmc_status st = TPMC_OK;
  for (int k = 0; k < 2 && st == TPMC_OK; ++k) {
    QueryDev q;
    if ((st = fill_query(m, params, each[k], &q)) != TPMC_OK) break;
    cudaEventRecord(tm.e0, c->stream);
    st = c->run(m, nullptr, kTrialDirs, &q, d_dirs, nullptr, nullptr, 0, (uint64_t)kTrialDirs * each[k],
                trace_variant(params, m.dev), (tpmc_result*)c->s_out.ptr, nullptr);
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
  const double dn = (double)kTrialDirs * (double)(each[1] - each[0]);
  *rate = (dn > 0.0 && dt > 0.0) ? dn / dt : (double)kTrialDirs * (double)each[1] / std::max((double)ms[1], 1e-6);
  return TPMC_OK;
}

// Best of two passes (the first also warms caches and clocks).
tpmc_status measure2(Ctx* c, const MeshRec& m, const tpmc_params* params, uint64_t N_trial, const double* d_dirs,
                     const LaunchCfg& cfg, bool manual, Timer& tm, double* rate, LaunchCfg* used) {
  double r0 = 0.0, r1 = 0.0;
  tpmc_status st = measure(c, m, params, N_trial, d_dirs, cfg, manual, tm, &r0, used);
  if (st == TPMC_OK) st = measure(c, m, params, N_trial, d_dirs, cfg, manual, tm, &r1, used);
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
  if ((st = c->grow(c->s_out, kTrialDirs * sizeof(tpmc_result), "results")) != TPMC_OK) return st;
  if ((st = c->grow(c->s_in, kTrialDirs * 3 * sizeof(double), "trial directions")) != TPMC_OK) return st;
  {
    double dirs[kTrialDirs * 3];
    trial_dirs(params, dirs);
    const cudaError_t e = cudaMemcpyAsync(c->s_in.ptr, dirs, sizeof(dirs), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tune directions");
  }
  const double* d_dirs = (const double*)c->s_in.ptr;
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
      st = measure2(c, *run_on, params, N_trial, d_dirs, LaunchCfg(), false, tm, &rate, nullptr);
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
  std::vector<std::pair<double, LaunchCfg>> scored;
  for (const LaunchCfg& cfg : cands) {
    double rate = 0.0;
    LaunchCfg used;
    if ((st = measure2(c, m, params, N_trial, d_dirs, cfg, true, tm, &rate, &used)) != TPMC_OK) return st;
    used.chunk = 0;
    scored.push_back({rate, used});
  }
  // the three best and the untuned schedule again on a four times longer
  // trial, so that a short trial's noise does not decide; the untuned
  // schedule is the one to beat, by 1 %
  std::sort(scored.begin(), scored.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
  const uint64_t N_long = std::min<uint64_t>(4 * N_trial, 1ull << 30);
  {
    double r = 0.0;
    LaunchCfg used;
    const auto had = c->tuned.find(tune_key(n_tri, variant));
    LaunchCfg kept;
    const bool had_tuned = had != c->tuned.end();
    if (had_tuned) { kept = had->second; c->tuned.erase(had); }
    st = measure2(c, m, params, N_long, d_dirs, LaunchCfg(), false, tm, &r, &used);
    if (had_tuned) c->tuned[tune_key(n_tri, variant)] = kept;
    if (st != TPMC_OK) return st;
    best_rate = 1.01 * r;
    best_cfg = used;
    best_cfg.chunk = 0;
  }
  for (size_t i = 0; i < scored.size() && i < 3; ++i) {
    double r = 0.0;
    LaunchCfg used;
    if ((st = measure2(c, m, params, N_long, d_dirs, scored[i].second, true, tm, &r, &used)) != TPMC_OK) return st;
    if (r > best_rate) {
      best_rate = r;
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
    if ((st = measure2(c, m, params, N_long, d_dirs, cfg, true, tm, &rate, &used)) != TPMC_OK) return st;
    if (rate > best_rate * 1.01) {  // a fixed chunk must beat the automatic one by more than the noise
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
