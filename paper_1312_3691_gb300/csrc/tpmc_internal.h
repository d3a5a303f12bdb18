// Internal layout shared by the host runtime (api.cpp, bvh.cpp, serve.cpp)
// and the CUDA kernels (kernels.cu).  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/tpmc.h"

namespace tpmc {

// Start tables of the inverse-CDF solves (they only start Newton's method;
// the root is then solved in the path's precision).  Both are laid out in
// z = Phi^-1(u), the standard normal quantile of the uniform, so that the
// tails are as finely resolved as the bulk.
// Latitude (Eq. 11), per query: x_j = H^-1(Phi(z_j)), z_j = kZLo + (kZHi - kZLo) j / kHTable.
constexpr int kHTable = 128;
constexpr double kZLo = -5.5, kZHi = 5.5;
// Normal speed (Eq. 14a), one table per context: x(s_i, z_j) with s_i = kVnSLo + i kVnStep
// (kVnNS rows, s in [-8, 16]) and z_j = kZLo + j kVnStep (kVnNZ columns); 69 KB.
constexpr double kVnSLo = -8.0, kVnStep = 0.125;
constexpr int kVnNS = 193, kVnNZ = 89;
// A queued particle keeps its id and query slot in one 64-bit word: ids
// below 2^40 (N <= 2^34) and at most 2^24 query slots per launch.
constexpr int kSlotPidBits = 40;
constexpr uint32_t kMaxLaunchQueries = 1u << 24;
constexpr int kMaxStack = 64;    // BVH traversal stack (the builder keeps depth below)
constexpr int kMaxRecordK = 64;  // hits recorded per particle in verification runs

// ---------------------------------------------------------------- mesh (device)
// Binary BVH node (32 bytes, both children's boxes in one node), boxes as
// 16-bit coordinates q on one grid over the whole mesh: along axis a the
// plane is qorigin[a] + q qstep[a] (qstep a power of two; the boxes are
// rounded outward and widened by one grid step, so float slab tests stay
// conservative).
//   words 0-2: child 0's (lo.x | hi.x << 16), (lo.y | hi.y << 16), (lo.z | hi.z << 16)
//   words 3-5: the same for child 1
//   words 6-7: child0, child1 as int.  child >= 0: inner node index;
//        child < 0: leaf ~(count << 24 | first), triangles [first, first+count)
//        of the leaf-ordered triangle arrays; count <= 127.
// Nodes are numbered breadth first, so nodes [0, k) are the top of the tree
// and can be staged in shared memory as a block.
constexpr int kBinaryNodeF4 = 2;  // float4 per binary node
// Compressed wide BVH node (after Ylitie, Karras & Laine, "Efficient
// incoherent ray traversal on GPUs through compressed wide BVHs", HPG 2017):
// the child boxes are 8-bit coordinates on a grid of the node's own, so one
// node fetch decides up to W children.  W = 8: 80 bytes (5 float4); W = 4:
// 64 bytes (4 float4).
//   w0 = (px, py, pz, e)  grid origin p (float); e: bytes ex, ey, ez (biased
//                         exponents: the grid step along axis a is 2^(ea - 127))
//                         and imask (bit s: slot s holds an inner node)
//   w1 = (child_base, tri_base, meta[0..3], meta[4..7] (W = 8 only))
//   then the planes qlo_x, qlo_y, qlo_z, qhi_x, qhi_y, qhi_z, one byte per
//   slot: W = 8: two words per plane (slots 0-3, 4-7) in w2.xyzw, w3.xyzw,
//   w4.xyzw; W = 4: one word per plane in w2.xyzw, w3.xy.
// Child box of slot s along axis a: [p_a + 2^e_a qlo_a[s], p_a + 2^e_a qhi_a[s]]
// (rounded outward from the padded float box); an empty slot has qlo = 255 >
// qhi = 0 on every axis.  Inner slot s: node child_base + (number of inner
// slots below s); children of a node are consecutive (breadth-first order).
// Leaf slot s: meta[s] = (count - 1) << 5 | offset, its triangles are
// tri_base + offset ... + count - 1 in the triangle arrays (count <= 4,
// offset + count <= 32: a node's leaf triangles form one block).
// Slot s of an 8-wide node lies towards the box corner s (bit 0: +x, bit 1:
// +y, bit 2: +z) of its parent; slot s of a 4-wide node towards corner
// kWide4Corner[s].  The traversal orders children by these corners.
constexpr int kWideLeafMax = 4;
constexpr int kMaxStackW = 32;     // wide traversal stack (the builder keeps the depth below)
constexpr uint32_t kWide4Corner[4] = {0u, 3u, 5u, 6u};

struct MeshDev {
  const float4* nodes = nullptr;    // binary: [n_nodes][4]; wide: [n_nodes][width == 8 ? 5 : 4]
  const float4* tris = nullptr;     // [n_tri_leaf][3]: (v0, id bits), (v1, 0), (v2, 0)
  const double* tris64 = nullptr;   // [n_tri_leaf][12]: v0, v1, v2, id, 0, 0
  const float4* frames = nullptr;   // [n_tri][2] by input index: (n, area), (t1, exposed-side bits)
  const double* frames64 = nullptr; // [n_tri][8] by input index: n, area, t1, exposed-side bits
  uint32_t n_nodes = 0;
  uint32_t n_tri = 0;               // input numbering (panel arrays use it)
  uint32_t n_tri_leaf = 0;          // triangles referenced by leaves (zero-area ones dropped)
  uint32_t width = 2;               // 2: binary nodes; 4 or 8: compressed wide nodes
  uint32_t depth = 0;               // levels below the root (bounds the wide traversal's stack)
  float scene_radius = 1.0f;
  // padded root box (empty: no mesh); binary trees: in grid units 2^23 + q
  float box_lo[3] = {0.0f, 0.0f, 0.0f}, box_hi[3] = {-1.0f, -1.0f, -1.0f};
  float qorigin[3] = {0.0f, 0.0f, 0.0f}, qstep[3] = {1.0f, 1.0f, 1.0f};  // grid of binary trees' boxes
};

// ------------------------------------------------------------- query (device)
// Layout of QueryDev::fc, the FP32 constants of a query.
enum : int {
  kFcS = 0, kFcCw = 1, kFcRcv = 2, kFcSqrtpi4S = 3,  // S, c_W / c_mp, CV radius, sqrt(pi) / (4 S)
  kFcK1 = 4, kFcDinv = 5, kFcScale = 6,              // latitude K1, 1 / D, fixed-point scale
  kFcR = 7,                                           // [9] Rodrigues matrix (Eq. 15), row major
  kFcCenter = 16, kFcVhat = 19, kFcRef = 22,          // [3] each
  kFcPole = 25,                                       // [6] latitude tail-mass cubics at x = +1, then -1
  kFcScale2 = 31,                                     // fixed-point scale of the squared drag contributions
  kFcCount = 32
};

// One query: inputs copied from tpmc_params, derived values written by the
// FP64 set-up kernel (flux normalisation, rotation, start table).
struct QueryDev {
  // inputs
  double n, T_inf, m, V, dir[3], T_W, eps, A_ref, ref[3], r_cv, center[3], l_ref;
  double rmax;            // bound on |hit point - ref| (mesh extent seen from ref)
  uint64_t N;             // particles of this query (ids 0..N-1)
  uint64_t seed;
  uint32_t stream_id, max_bounces;
  uint32_t precision;
  uint32_t cv_kind;       // TPMC_CV_*
  double box_lo[3], box_hi[3];
  uint32_t gsi_model;     // TPMC_GSI_*
  uint32_t eps_k;         // Maxwell: diffuse iff the top 23 bits k of the draw satisfy k < eps_k, which
                          // is u = (k + 1/2) 2^-23 < eps exactly (eps_k = ceil(eps 2^23 - 1/2))
  double cll[4];          // CLL: alpha_n, sqrt(1 - alpha_n), alpha_t = sigma_t (2 - sigma_t), sqrt(1 - alpha_t)
  float fcll[4];
  long long* panel;       // [n_tri][3] fixed-point per-triangle sums, or null
  // derived by the set-up kernel
  double S, cw, c_mp, gamma, q_inf, Dnorm, K1, vhat[3], R[9];
  double quantum;         // 2^-shift
  double quantum2;        // 2^-shift2: unit of the sum of squared drag contributions
  int32_t shift;          // fixed-point scale 2^shift
  int32_t shift2;         // fixed-point scale of the squared drag contributions
  int32_t status;         // tpmc_status of the set-up
  int32_t pad2;
  // FP32 copies of the query constants (kFc* indices)
  float fc[kFcCount];
  float htab[kHTable + 1];
  // box CV (cv_kind != sphere): face f = 2a + k is x_a = hi_a (k = 0) or lo_a
  // (k = 1) and owns particle ids [face_end[f-1], face_end[f]); s_f is its
  // inward-normal speed ratio
  uint64_t face_end[6];
  double face_s[6];
  float fface_s[6], fbox_lo[3], fbox_ext[3];
};

// Work item: particles [pid_begin, pid_begin + count) of query `query`,
// occupying global work indices [g_begin, g_begin + count).
struct ItemDev {
  uint64_t g_begin;
  uint64_t pid_begin;
  uint64_t count;
  uint32_t query;
  uint32_t pad;
};

// Per-query accumulators (device, zeroed before a launch).
// One query's integer sums, kept as kAccStripes copies ("stripes") of one
// 128-byte line each: a warp adds to the stripe its index selects, so when a
// whole grid moves on to the next query its atomics spread over several L2
// slices instead of queueing on one line.  The array is stripe-major: stripe
// j of query q is acc[j * stride + q], stride being the array's number of
// query slots, so a query's stripes lie stride * 128 bytes apart wherever the
// array starts (with a query's stripes in one 1 KB block the launches ran
// 15-35 % slower at one alignment of the block than at the other).  The final
// reduction adds the stripes (integer sums, so the split changes no result).
constexpr int kAccStripes = 8;
struct alignas(128) AccStripe {
  long long F[3];           // sum of (v_in - v_out), units quantum * c_mp
  long long T[3];           // sum of (r - ref) x (v_in - v_out), units quantum * m * c_mp
  unsigned long long hits, hit_particles, truncated, particles, nodes, tris;
  // sum over particles of (their dv . Vhat)^2 in units of quantum2, as three
  // limbs of one 128-bit integer, d2[0] + d2[1] 2^30 + d2[2] 2^60: each flush
  // adds bits 0-29 and 30-59 of its sum to the first two and the rest to the
  // third, with atomics that return nothing.  The total is exact and does not
  // depend on the order of the flushes; the limbs alone do.
  unsigned long long d2[3];
  unsigned long long pad;
};
static_assert(sizeof(AccStripe) == 128, "one stripe per 128-byte line");

struct RecordsDev {
  double* pos = nullptr;
  double* vel = nullptr;
  double* dv = nullptr;
  uint32_t* n_hits = nullptr;
  uint32_t* truncated = nullptr;
  uint32_t* tri = nullptr;
  uint32_t K = 0;
};

struct TraceArgs {
  MeshDev mesh;
  const QueryDev* queries;
  AccStripe* acc;             // stripe-major: stripe j of query q at acc[j * acc_stride + q]
  uint32_t acc_stride;
  const ItemDev* items;
  uint32_t n_items;
  uint32_t chunk;             // ids a warp takes per fetch
  uint32_t smem_nodes;        // nodes staged in shared memory
  uint32_t count_work;        // 1: count node visits and triangle tests
  uint32_t refill_at;         // finished lanes that end a traversal round
  uint64_t total;             // sum of item counts
  unsigned long long* counter;  // global work counter (zeroed before launch)
  int* error;                 // device error word (stack overflow)
  const float* vn_table;      // [kVnNS][kVnNZ] normal-speed start table
  RecordsDev rec;
};

struct LaunchCfg {
  uint32_t block = 128;
  uint32_t blocks_per_sm = 4;
  uint32_t chunk = 0;
  uint32_t smem_nodes = 0;
  uint32_t refill_at = 0;      // 0: the default (16)
};

// ------------------------------------------------------------ host launchers
// Trace-kernel variant: the precision (TPMC_FP32 / TPMC_FP64), plus
// kVariantCll when the launch holds a query with the CLL surface model (so
// that launches without one run code compiled without that branch), plus the
// mesh's BVH layout (kVariantWide4 / kVariantWide8 for compressed wide nodes),
// plus kVariantCount when the launch counts node visits and triangle tests or
// writes per-particle records (launches that do neither run code without the
// two counters and without each particle's momentum-change vector, which the
// 64-register build otherwise keeps live through the traversal loop).
constexpr uint32_t kVariantCll = 2u;
constexpr uint32_t kVariantWide4 = 4u, kVariantWide8 = 8u;
constexpr uint32_t kVariantCount = 16u;
inline uint32_t trace_variant(const tpmc_params* p, const MeshDev& m) {
  return p->precision | (p->gsi_model == TPMC_GSI_CLL ? kVariantCll : 0u) |
         (m.width == 8 ? kVariantWide8 : (m.width == 4 ? kVariantWide4 : 0u));
}
inline uint32_t variant_width(uint32_t v) { return (v & kVariantWide8) ? 8u : ((v & kVariantWide4) ? 4u : 2u); }
inline uint32_t node_float4s(uint32_t width) { return width == 8 ? 5u : (width == 4 ? 4u : 2u); }

// Set-up of nq queries (block i: slot slots[i], or i), which also clears
// their accumulator stripes in acc (stripe-major, acc_stride slots per stripe).
cudaError_t launch_setup(QueryDev* d_queries, uint32_t nq, const QueryDev* d_base, const double* d_dirs,
                         const double* d_S, ItemDev* d_items, const uint32_t* d_slots, AccStripe* d_acc,
                         uint32_t acc_stride, cudaStream_t stream);
cudaError_t launch_vn_table(float* d_table, cudaStream_t stream);
cudaError_t launch_trace(const TraceArgs& args, uint32_t variant, const LaunchCfg& cfg, int num_sms,
                         cudaStream_t stream);
cudaError_t launch_finalize(const QueryDev* d_queries, const AccStripe* d_acc, uint32_t acc_stride, uint32_t nq,
                            const uint32_t* d_slots, tpmc_result* d_out, cudaStream_t stream);
cudaError_t launch_panels(const QueryDev* d_query, const long long* d_panel, const float4* frames,
                          const double* frames64, uint32_t n_tri, double* d_pressure, double* d_shear,
                          cudaStream_t stream);
size_t trace_smem_bytes(const LaunchCfg& cfg, uint32_t n_nodes, uint32_t variant);
int trace_max_blocks_per_sm(uint32_t variant, const LaunchCfg& cfg, uint32_t n_nodes);

// ---------------------------------------------------------------- BVH (host)
struct BvhBuild {
  std::size_t n_nodes = 0;
  uint32_t width = 2;        // children per node: 2 (binary layout) or 4, 8 (compressed wide layout)
  uint32_t node_bytes = 64;  // bytes per node in `nodes`
  float root_lo[3] = {0.0f, 0.0f, 0.0f}, root_hi[3] = {-1.0f, -1.0f, -1.0f};  // padded root box (empty: no mesh)
  // binary layout: the boxes' grid, and the root box in grid units 2^23 + q
  float qorigin[3] = {0.0f, 0.0f, 0.0f}, qstep[3] = {1.0f, 1.0f, 1.0f};
  float qroot_lo[3] = {0.0f, 0.0f, 0.0f}, qroot_hi[3] = {-1.0f, -1.0f, -1.0f};
  uint32_t depth = 0, leaf_max = 0, n_skipped = 0;
  uint32_t n_exposed = 0;    // triangle sides the whole mesh lies behind
  // host copies ready for upload
  float* nodes = nullptr;    // [n_nodes * node_bytes / 4]
  float* tris = nullptr;     // [n_leaf_tris * 12]
  double* tris64 = nullptr;  // [n_leaf_tris * 12]
  float* frames = nullptr;   // [n_tri * 8]: n, area, t1, exposed-side bits (uint32 in word 7)
  double* frames64 = nullptr;// [n_tri * 8]: n, area, t1, exposed-side bits (as a double in word 7)
  uint32_t n_leaf_tris = 0;
  double center[3] = {0, 0, 0}, radius = 0;
  void release();
};

// Builds a BVH over the mesh by the surface-area heuristic with spatial
// splits and lays it out with `width` children per node (2: binary nodes;
// 4 or 8: compressed wide nodes collapsed from the binary tree).  Returns
// false (with a message) on invalid input.
bool build_bvh(const double* xyz, uint32_t n_vert, const uint32_t* tri, uint32_t n_tri, uint32_t max_leaf,
               uint32_t width, BvhBuild* out, const char** err);

}  // namespace tpmc
