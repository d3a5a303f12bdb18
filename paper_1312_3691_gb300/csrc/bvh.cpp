// Host-side bounding-volume hierarchy for closest-hit ray tracing.
//
// The paper represents the spacecraft by a triangulation and relies on
// "well-known ray-tracing methods" for the closest intersection (§II.A); it
// does not name a structure.  This builder makes a binary BVH by binned
// surface-area heuristic (16 bins per axis), then lays it out for the GPU:
// each node carries both children's boxes (one 64-byte fetch decides both),
// nodes are numbered breadth first so that the top k nodes form a block that
// the trace kernel stages in shared memory, and triangles are stored in leaf
// order (48 bytes each in float, 96 in double).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <vector>

#include "tpmc_internal.h"

namespace tpmc {

void BvhBuild::release() {
  std::free(nodes); std::free(tris); std::free(tris64); std::free(frames); std::free(frames64);
  nodes = tris = frames = nullptr;
  tris64 = frames64 = nullptr;
}

namespace {

struct Box {
  double lo[3] = {INFINITY, INFINITY, INFINITY};
  double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const double p[3]) {
    for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], p[a]); hi[a] = std::max(hi[a], p[a]); }
  }
  void grow(const Box& b) {
    for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], b.lo[a]); hi[a] = std::max(hi[a], b.hi[a]); }
  }
  bool empty() const { return !(lo[0] <= hi[0]); }
  double area() const {
    if (empty()) return 0.0;
    const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return 2.0 * (dx * dy + dy * dz + dz * dx);
  }
};

struct Prim {
  Box box;
  double c[3];
  uint32_t id;
};

struct BNode {       // binary build node
  Box box;
  int32_t left = -1, right = -1;  // children (build indices) for inner nodes
  uint32_t first = 0, count = 0;  // leaf range in prims
  uint32_t depth = 0;
};

constexpr int kBins = 16;
constexpr double kCostNode = 1.0;
constexpr double kCostTri = 1.2;
constexpr uint32_t kMaxDepth = kMaxStack - 20;  // SAH below this depth, median splits after

}  // namespace

bool build_bvh(const double* xyz, uint32_t n_vert, const uint32_t* tri, uint32_t n_tri, uint32_t max_leaf,
               BvhBuild* out, const char** err) {
  *out = BvhBuild();
  max_leaf = std::max(1u, std::min(max_leaf, 127u));
  if (n_tri > (1u << 24)) { *err = "mesh has more than 2^24 triangles"; return false; }
  if (n_tri > 0 && n_vert == 0) { *err = "triangles without vertices"; return false; }
  for (uint64_t i = 0; i < (uint64_t)n_vert * 3; ++i)
    if (!std::isfinite(xyz[i])) { *err = "non-finite vertex coordinate"; return false; }
  for (uint64_t i = 0; i < (uint64_t)n_tri * 3; ++i)
    if (tri[i] >= n_vert) { *err = "triangle vertex index out of range"; return false; }

  // bounding sphere: centre of the box of the referenced vertices, largest distance
  Box all;
  for (uint64_t i = 0; i < (uint64_t)n_tri * 3; ++i) all.grow(xyz + 3 * (uint64_t)tri[i]);
  if (!all.empty()) {
    for (int a = 0; a < 3; ++a) out->center[a] = 0.5 * (all.lo[a] + all.hi[a]);
    double r2 = 0;
    for (uint64_t i = 0; i < (uint64_t)n_tri * 3; ++i) {
      const double* p = xyz + 3 * (uint64_t)tri[i];
      double d2 = 0;
      for (int a = 0; a < 3; ++a) d2 += (p[a] - out->center[a]) * (p[a] - out->center[a]);
      r2 = std::max(r2, d2);
    }
    out->radius = std::sqrt(r2);
  }
  const double scale = std::max(out->radius, 1e-6);

  // per-triangle frame by input index (normal, area, unit first edge)
  out->frames = (float*)std::calloc((size_t)std::max(n_tri, 1u) * 8, sizeof(float));
  out->frames64 = (double*)std::calloc((size_t)std::max(n_tri, 1u) * 8, sizeof(double));
  std::vector<Prim> prims;
  prims.reserve(n_tri);
  for (uint32_t i = 0; i < n_tri; ++i) {
    const double* a = xyz + 3 * (uint64_t)tri[3 * i];
    const double* b = xyz + 3 * (uint64_t)tri[3 * i + 1];
    const double* c = xyz + 3 * (uint64_t)tri[3 * i + 2];
    const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double cn = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    const double el = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    double* f64 = out->frames64 + 8 * (size_t)i;
    float* f32 = out->frames + 8 * (size_t)i;
    if (!(cn > 0.0) || !(el > 0.0)) { ++out->n_skipped; continue; }
    for (int k = 0; k < 3; ++k) { f64[k] = cr[k] / cn; f64[4 + k] = e1[k] / el; }
    f64[3] = 0.5 * cn;
    for (int k = 0; k < 8; ++k) f32[k] = (float)f64[k];
    Prim p;
    p.box.grow(a); p.box.grow(b); p.box.grow(c);
    for (int k = 0; k < 3; ++k) p.c[k] = (a[k] + b[k] + c[k]) / 3.0;
    p.id = i;
    prims.push_back(p);
  }

  // ---- binned SAH build (iterative) ----
  std::vector<BNode> bn;
  bn.reserve(2 * prims.size() / std::max(1u, max_leaf / 2) + 4);
  std::vector<int32_t> todo;
  if (!prims.empty()) {
    BNode root;
    root.first = 0; root.count = (uint32_t)prims.size();
    for (const Prim& p : prims) root.box.grow(p.box);
    bn.push_back(root);
    todo.push_back(0);
  }
  std::vector<Prim> tmp;
  while (!todo.empty()) {
    const int32_t ni = todo.back();
    todo.pop_back();
    BNode nd = bn[ni];
    const uint32_t first = nd.first, count = nd.count;
    // centroid bounds
    Box cb;
    for (uint32_t k = first; k < first + count; ++k) cb.grow(prims[k].c);
    int best_axis = -1, best_bin = -1;
    double best_cost = INFINITY;
    if (count > 1) {
      for (int a = 0; a < 3; ++a) {
        const double ext = cb.hi[a] - cb.lo[a];
        if (!(ext > 0.0)) continue;
        Box bins[kBins];
        uint32_t cnt[kBins] = {0};
        for (uint32_t k = first; k < first + count; ++k) {
          int b = (int)((prims[k].c[a] - cb.lo[a]) / ext * kBins);
          b = std::min(std::max(b, 0), kBins - 1);
          bins[b].grow(prims[k].box);
          ++cnt[b];
        }
        Box lbox[kBins], rbox[kBins];
        uint32_t lcnt[kBins], rcnt[kBins];
        Box acc; uint32_t c = 0;
        for (int b = 0; b < kBins; ++b) { acc.grow(bins[b]); c += cnt[b]; lbox[b] = acc; lcnt[b] = c; }
        acc = Box(); c = 0;
        for (int b = kBins - 1; b >= 0; --b) { acc.grow(bins[b]); c += cnt[b]; rbox[b] = acc; rcnt[b] = c; }
        for (int b = 0; b + 1 < kBins; ++b) {
          if (lcnt[b] == 0 || rcnt[b + 1] == 0) continue;
          const double cost = kCostNode + kCostTri * (lbox[b].area() * lcnt[b] + rbox[b + 1].area() * rcnt[b + 1]) /
                                              std::max(nd.box.area(), 1e-300);
          if (cost < best_cost) { best_cost = cost; best_axis = a; best_bin = b; }
        }
      }
    }
    const double leaf_cost = kCostTri * count;
    const bool must_split = count > max_leaf;
    bool make_leaf = count <= 1 || nd.depth >= kMaxDepth || (!must_split && best_cost >= leaf_cost);
    uint32_t mid = first;
    if (!make_leaf) {
      if (best_axis >= 0) {
        const double ext = cb.hi[best_axis] - cb.lo[best_axis];
        auto is_left = [&](const Prim& p) {
          int b = (int)((p.c[best_axis] - cb.lo[best_axis]) / ext * kBins);
          b = std::min(std::max(b, 0), kBins - 1);
          return b <= best_bin;
        };
        mid = (uint32_t)(std::partition(prims.begin() + first, prims.begin() + first + count, is_left) -
                         prims.begin());
      }
      if (mid == first || mid == first + count) {
        // all centroids coincide (or no useful bin): split the range in half
        mid = first + count / 2;
      }
      if (count > max_leaf && nd.depth >= kMaxDepth) make_leaf = true;
    }
    if (make_leaf) {
      if (count > 127) {
        // depth limit reached with an oversized leaf: split by median regardless
        mid = first + count / 2;
      } else {
        bn[ni].left = bn[ni].right = -1;
        continue;
      }
    }
    BNode l, r;
    l.first = first; l.count = mid - first; l.depth = nd.depth + 1;
    r.first = mid; r.count = first + count - mid; r.depth = nd.depth + 1;
    for (uint32_t k = l.first; k < l.first + l.count; ++k) l.box.grow(prims[k].box);
    for (uint32_t k = r.first; k < r.first + r.count; ++k) r.box.grow(prims[k].box);
    const int32_t li = (int32_t)bn.size();
    bn.push_back(l);
    const int32_t ri = (int32_t)bn.size();
    bn.push_back(r);
    bn[ni].left = li;
    bn[ni].right = ri;
    todo.push_back(ri);
    todo.push_back(li);
  }

  // ---- GPU layout: inner nodes in breadth-first order, leaves in place ----
  // A tree that is a single leaf gets a root whose second child is empty.
  std::vector<int32_t> inner_order;  // build index of each GPU node
  std::vector<int32_t> gpu_index(bn.size(), -1);
  std::vector<uint32_t> gpu_depth;
  bool single_leaf = !bn.empty() && bn[0].left < 0;
  if (!bn.empty() && !single_leaf) {
    std::deque<int32_t> q;
    q.push_back(0);
    while (!q.empty()) {
      const int32_t b = q.front();
      q.pop_front();
      gpu_index[b] = (int32_t)inner_order.size();
      inner_order.push_back(b);
      for (int32_t c : {bn[b].left, bn[b].right})
        if (bn[c].left >= 0) q.push_back(c);
    }
  }
  const size_t n_nodes = bn.empty() ? 0 : (single_leaf ? 1 : inner_order.size());
  out->n_nodes = n_nodes;
  out->nodes = (float*)std::calloc(std::max<size_t>(n_nodes, 1) * 16, sizeof(float));

  // triangles in leaf order
  out->n_leaf_tris = (uint32_t)prims.size();
  out->tris = (float*)std::calloc(std::max<size_t>(prims.size(), 1) * 12, sizeof(float));
  out->tris64 = (double*)std::calloc(std::max<size_t>(prims.size(), 1) * 12, sizeof(double));
  for (size_t k = 0; k < prims.size(); ++k) {
    const uint32_t i = prims[k].id;
    for (int v = 0; v < 3; ++v) {
      const double* p = xyz + 3 * (uint64_t)tri[3 * i + v];
      for (int a = 0; a < 3; ++a) {
        out->tris[12 * k + 4 * v + a] = (float)p[a];
        out->tris64[12 * k + 3 * v + a] = p[a];
      }
    }
    uint32_t idbits = i;
    std::memcpy(&out->tris[12 * k + 3], &idbits, 4);
    out->tris64[12 * k + 9] = (double)i;
  }

  // conservative float boxes: pad by a small multiple of the scene scale and
  // of the coordinate, then round outward
  auto pad_lo = [&](double v) {
    const double p = v - (1e-5 * scale + 4e-7 * std::fabs(v));
    float f = (float)p;
    if ((double)f > p) f = std::nextafter(f, -INFINITY);
    return f;
  };
  auto pad_hi = [&](double v) {
    const double p = v + (1e-5 * scale + 4e-7 * std::fabs(v));
    float f = (float)p;
    if ((double)f < p) f = std::nextafter(f, INFINITY);
    return f;
  };
  auto child_code = [&](int32_t b, uint32_t& depth_seen) -> int32_t {
    const BNode& c = bn[b];
    depth_seen = std::max(depth_seen, c.depth);
    if (c.left >= 0) return gpu_index[b];
    out->leaf_max = std::max(out->leaf_max, c.count);
    return ~(int32_t)((c.count << 24) | c.first);
  };
  auto write_child = [&](float* nd, int slot, const Box* box) {
    // slot 0 -> n0 and n2.xy ; slot 1 -> n1 and n2.zw
    float* xy = nd + 4 * slot;
    float* z = nd + 8 + 2 * slot;
    if (box == nullptr) {
      // empty child: a point box far outside any control volume, which no ray reaches
      xy[0] = xy[1] = xy[2] = xy[3] = z[0] = z[1] = 1e30f;
      return;
    }
    xy[0] = pad_lo(box->lo[0]); xy[1] = pad_hi(box->hi[0]);
    xy[2] = pad_lo(box->lo[1]); xy[3] = pad_hi(box->hi[1]);
    z[0] = pad_lo(box->lo[2]); z[1] = pad_hi(box->hi[2]);
  };
  uint32_t depth_seen = 0;
  if (single_leaf) {
    float* nd = out->nodes;
    write_child(nd, 0, &bn[0].box);
    write_child(nd, 1, nullptr);
    int32_t c0 = child_code(0, depth_seen), c1 = ~(int32_t)0;  // empty leaf: count 0
    std::memcpy(nd + 12, &c0, 4);
    std::memcpy(nd + 13, &c1, 4);
  } else {
    for (size_t g = 0; g < inner_order.size(); ++g) {
      const BNode& b = bn[inner_order[g]];
      float* nd = out->nodes + 16 * g;
      write_child(nd, 0, &bn[b.left].box);
      write_child(nd, 1, &bn[b.right].box);
      int32_t c0 = child_code(b.left, depth_seen), c1 = child_code(b.right, depth_seen);
      std::memcpy(nd + 12, &c0, 4);
      std::memcpy(nd + 13, &c1, 4);
    }
  }
  out->depth = depth_seen;
  if (out->depth + 1 >= (uint32_t)kMaxStack) {
    out->release();
    *err = "bounding-volume hierarchy deeper than the traversal stack";
    return false;
  }
  return true;
}

}  // namespace tpmc
