// Autotuner of the trace kernel's launch schedule.
//
// Candidates: threads per block, shared-memory BVH nodes, resident blocks per
// SM (the highest occupancy, 6 and 4) and the traversal-round refill threshold.  Each is timed with CUDA events on a short run of
// the caller's query; the fastest is kept for the mesh's size class (powers of
// 4 of the triangle count) and kernel variant, and later launches on meshes of that
// class use it.
#include <algorithm>
#include <cstring>
#include <vector>

#include "runtime.h"

using namespace tpmc;

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
  const MeshRec& m = it->second;
  cudaSetDevice(c->device);
  QueryDev q;
  if ((st = fill_query(m, params, N_trial, &q)) != TPMC_OK) return st;
  ItemDev item;
  std::memset(&item, 0, sizeof(item));
  item.count = N_trial;
  if ((st = c->grow(c->s_out, sizeof(tpmc_result), "result")) != TPMC_OK) return st;

  std::vector<LaunchCfg> cands;
  const uint32_t nn = m.dev.n_nodes;
  for (uint32_t block : {64u, 128u, 256u})
    for (uint32_t sm_nodes : {0u, 256u}) {
      for (uint32_t occ : {0u, 6u, 4u})  // 0: the highest occupancy
        for (uint32_t refill : {8u, 16u, 24u}) {
          LaunchCfg cfg;
          cfg.block = block;
          cfg.smem_nodes = std::min(sm_nodes, nn);
          cfg.refill_at = refill;
          const int maxb = trace_max_blocks_per_sm(trace_variant(params), cfg, nn);
          if (maxb < 1 || (occ != 0 && occ >= (uint32_t)maxb)) continue;
          cfg.blocks_per_sm = occ == 0 ? (uint32_t)maxb : occ;
          cfg.chunk = 0;
          cands.push_back(cfg);
        }
    }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bool had_manual = c->manual_launch;
  const LaunchCfg old_manual = c->manual;
  // Each candidate runs a quarter of N_trial and then all of it; the score is
  // the marginal rate (N_trial - N_trial / 4) / (t_full - t_quarter), so the
  // fixed costs of a launch (set-up, reduction, the tail of its last warps)
  // drop out and the choice holds for the long launches of sweeps.  The
  // chunk stays automatic, so each later launch sizes it from its own total.
  const uint64_t quarter = std::max<uint64_t>(1, N_trial / 4);
  double best_rate = -1.0;
  LaunchCfg best_cfg;
  for (int pass = 0; pass < 2; ++pass) {  // pass 0 warms caches and clocks
    for (const LaunchCfg& cfg : cands) {
      c->manual_launch = true;
      c->manual = cfg;
      float ms[2] = {0.0f, 0.0f};
      LaunchCfg used;
      for (int k = 0; k < 2 && st == TPMC_OK; ++k) {
        item.count = k == 0 ? quarter : N_trial;
        cudaEventRecord(e0, c->stream);
        st = c->run(m, &q, 1, nullptr, nullptr, nullptr, &item, 1, item.count, trace_variant(params),
                    (tpmc_result*)c->s_out.ptr, nullptr);
        cudaEventRecord(e1, c->stream);
        if (st != TPMC_OK) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { st = cuda_fail(e, "tune"); break; }
        cudaEventElapsedTime(&ms[k], e0, e1);
        used = c->last_cfg;
      }
      if (st != TPMC_OK) break;
      const double dt = (double)ms[1] - (double)ms[0];
      const double rate = (N_trial > quarter && dt > 0.0) ? (double)(N_trial - quarter) / dt
                                                          : (double)N_trial / std::max((double)ms[1], 1e-6);
      if (pass == 1 && rate > best_rate) {
        best_rate = rate;
        best_cfg = used;
        best_cfg.chunk = 0;
      }
    }
    if (st != TPMC_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->manual_launch = had_manual;
  c->manual = old_manual;
  if (st != TPMC_OK) return st;
  if ((st = c->check_error_word()) != TPMC_OK) return st;
  c->tuned[tune_key(m.dev.n_tri, trace_variant(params))] = best_cfg;
  if (best) {
    best->block = best_cfg.block;
    best->blocks_per_sm = best_cfg.blocks_per_sm;
    best->chunk = best_cfg.chunk;
    best->smem_nodes = best_cfg.smem_nodes;
    best->refill_at = best_cfg.refill_at;
    best->bvh_leaf = c->bvh_leaf;
  }
  return TPMC_OK;
}
