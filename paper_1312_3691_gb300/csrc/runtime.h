// Host-side context of the TPMC library (not part of the ABI).
#pragma once

#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "tpmc_internal.h"

namespace tpmc {

extern thread_local std::string g_last_error;
tpmc_status fail(tpmc_status st, const std::string& msg);
tpmc_status cuda_fail(cudaError_t e, const char* where);
tpmc_status validate_params(const tpmc_params* p);

struct MeshRec {
  MeshDev dev;
  void* d_block = nullptr;     // one device allocation holding every mesh array
  size_t bytes = 0;
  double center[3] = {0, 0, 0}, radius = 0;
  uint32_t depth = 0, leaf_max = 0, n_skipped = 0, n_vert = 0, n_exposed = 0, node_bytes = 64;
  std::vector<double> h_xyz;   // host copy for the control-volume containment check
  std::vector<uint32_t> h_tri;
  int in_use = 0;              // queries in flight on this mesh (serving)
};

struct PanelRec {
  void* d_panel = nullptr;     // [n_tri][3] int64 fixed-point sums
  QueryDev query;              // set-up values needed for the conversion
  tpmc_mesh_id mesh = 0;
  uint32_t n_tri = 0;
};

struct Scratch {
  void* ptr = nullptr;
  size_t cap = 0;
};

struct ServeState;  // serve.cpp

// BVH width of mesh loads that neither tpmc_set_launch nor tpmc_tune decided.
constexpr uint32_t kDefaultBvhWidth = 2;

tpmc_status fill_query(const MeshRec& m, const tpmc_params* p, uint64_t N, QueryDev* q);

inline uint64_t tune_key(uint32_t n_tri, uint32_t variant) {
  // size classes: powers of 4 of the triangle count; one table per kernel variant
  uint32_t cls = 0;
  while (n_tri > 1 && cls < 16) { n_tri >>= 2; ++cls; }
  return ((uint64_t)variant << 32) | cls;
}

struct Ctx {
  int device = 0;
  int num_sms = 1;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  size_t budget = 0, used = 0;
  uint64_t n_allocs = 0;       // device allocations made since creation
  std::map<void*, size_t> sizes;
  std::recursive_mutex mu;
  std::map<tpmc_mesh_id, MeshRec> meshes;
  tpmc_mesh_id next_mesh = 1;
  std::map<tpmc_query_id, PanelRec> panels;
  tpmc_query_id next_query = 1;
  bool counters = false;
  bool manual_launch = false;
  uint32_t bvh_leaf = 4;       // largest leaf of the BVHs built by later mesh loads
  uint32_t bvh_width = 0;      // children per node of later mesh loads (0: tuned or default)
  std::map<uint64_t, uint32_t> tuned_width;  // BVH width chosen by tpmc_tune per size class
  LaunchCfg manual;
  LaunchCfg last_cfg;
  std::map<uint64_t, LaunchCfg> tuned;
  Scratch s_queries, s_acc, s_items, s_misc, s_base, s_out, s_in;
  float* vn_table = nullptr;   // normal-speed start table, built once at creation
  void* h_pinned = nullptr;
  int* h_err_word = nullptr;
  ServeState* serve = nullptr;

  uint32_t width_for(uint32_t n_tri) const;
  tpmc_status upload_mesh(const double* xyz, uint32_t n_vert, const uint32_t* tri, uint32_t n_tri, uint32_t width,
                          MeshRec* out);
  tpmc_status alloc(void** p, size_t bytes, const char* what);
  void release(void* p);
  tpmc_status grow(Scratch& s, size_t bytes, const char* what);
  LaunchCfg schedule(const MeshRec& m, uint32_t variant, uint64_t total);  // variant: see trace_variant
  tpmc_status run(const MeshRec& m, const QueryDev* h_queries, uint32_t nq, const QueryDev* h_base,
                  const double* d_dirs, const double* d_S, const ItemDev* h_items, uint32_t n_items,
                  uint64_t total, uint32_t variant, tpmc_result* d_out, const RecordsDev* rec);
  tpmc_status check_error_word();
  ~Ctx();
};

void stop_serving(Ctx* c);
// Wakes the serving scheduler after device memory was released outside it
// (panel loads read by tpmc_panels), so that queries waiting for memory retry.
void serve_memory_released(Ctx* c);

}  // namespace tpmc
