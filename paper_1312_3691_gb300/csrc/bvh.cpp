// Host-side bounding-volume hierarchy for closest-hit ray tracing.
//
// The paper represents the spacecraft by a triangulation and relies on
// "well-known ray-tracing methods" for the closest intersection (§II.A); it
// does not name a structure.  This builder makes a binary BVH by the surface
// area heuristic with spatial splits (Stich, Friedrich & Dietrich, "Spatial
// splits in bounding volume hierarchies", HPG 2009): besides binned object
// splits it considers planes that cut triangles, so that a triangle may be
// referenced by several leaves, each with the box of its part on that side.
// Long thin triangles that meet at a point (the fans that close a cylinder or
// a dish) otherwise give boxes that all overlap there.  Then it lays the tree
// out for the GPU: each node carries both children's boxes (one 64-byte fetch
// decides both), nodes are numbered breadth first so that the top k nodes
// form a block that the trace kernel stages in shared memory, and triangle
// references are stored in leaf order (48 bytes each in float, 96 in double).
//
// A closest hit stays exact: the parts of a triangle cover it, every part's
// box contains its part, so the ray meets the box of the part that holds the
// hit point no later than the hit, and ties between references of one
// triangle compare equal.
//
// It also marks each triangle side that the whole mesh lies behind (every
// face of a convex body, both sides of a flat sheet): a particle re-emitted
// from such a side has nothing ahead of it, so the trace kernel skips its
// traversal.  The marks go in the spare word of the triangle's frame.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <thread>
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
  const double* v[3];  // vertices
  uint32_t id;
};

// A reference to prims[p] restricted to `box` (a part of its bounding box).
struct Ref {
  Box box;
  uint32_t p;
};

Box intersect(const Box& a, const Box& b) {
  Box r;
  for (int k = 0; k < 3; ++k) {
    r.lo[k] = std::max(a.lo[k], b.lo[k]);
    r.hi[k] = std::min(a.hi[k], b.hi[k]);
  }
  for (int k = 0; k < 3; ++k)
    if (!(r.lo[k] <= r.hi[k])) return Box();
  return r;
}

// Splits the part of triangle `t` inside `box` by the plane x_axis = plane:
// the boxes of the polygon's vertices and edge crossings on each side,
// clipped to `box`.  Either side may come back empty.
void split_ref(const Prim& t, const Box& box, int axis, double plane, Box& left, Box& right) {
  left = Box();
  right = Box();
  for (int i = 0; i < 3; ++i) {
    const double* a = t.v[i];
    const double* b = t.v[(i + 1) % 3];
    if (a[axis] <= plane) left.grow(a);
    if (a[axis] >= plane) right.grow(a);
    if ((a[axis] < plane && b[axis] > plane) || (a[axis] > plane && b[axis] < plane)) {
      const double s = (plane - a[axis]) / (b[axis] - a[axis]);
      double x[3];
      for (int k = 0; k < 3; ++k) x[k] = a[k] + s * (b[k] - a[k]);
      x[axis] = plane;
      left.grow(x);
      right.grow(x);
    }
  }
  if (!left.empty()) left.hi[axis] = std::min(left.hi[axis], plane);
  if (!right.empty()) right.lo[axis] = std::max(right.lo[axis], plane);
  left = intersect(left, box);
  right = intersect(right, box);
}

// Grows bins[b], b0 <= b <= b1, by the box of the part of triangle `t` inside
// `box` that lies in slab b, [lo + b w, lo + (b + 1) w] along `axis` (the
// first and last slab open outwards): the box of the triangle's vertices and
// of its edges' crossings with the planes between the slabs.  A vertex on a
// plane counts on both sides of it.
void add_parts(const Prim& t, const Box& box, int axis, double lo, double w, int b0, int b1, Box* bins) {
  Box part[32];
  for (int i = 0; i < 3; ++i) {
    const double* p = t.v[i];
    const double* q = t.v[(i + 1) % 3];
    const int bp = std::min(std::max((int)((p[axis] - lo) / w), b0), b1);
    part[bp - b0].grow(p);
    const double pa = p[axis], qa = q[axis];
    if (pa == qa) continue;
    const double e_lo = std::min(pa, qa), e_hi = std::max(pa, qa);
    for (int b = b0; b < b1; ++b) {
      const double x = lo + (b + 1) * w;
      if (x < e_lo || x > e_hi) continue;
      const double s = (x - pa) / (qa - pa);
      double c[3];
      for (int k = 0; k < 3; ++k) c[k] = p[k] + s * (q[k] - p[k]);
      c[axis] = x;
      part[b - b0].grow(c);
      part[b + 1 - b0].grow(c);
    }
  }
  for (int b = b0; b <= b1; ++b) {
    Box& pb = part[b - b0];
    if (pb.empty()) continue;
    if (b > b0) pb.lo[axis] = std::max(pb.lo[axis], lo + b * w);
    if (b < b1) pb.hi[axis] = std::min(pb.hi[axis], lo + (b + 1) * w);
    bins[b].grow(intersect(pb, box));
  }
}

// Largest (sign = +1) or smallest (sign = -1) value of n . (x - o) over box b.
double box_extreme(const Box& b, const double n[3], const double o[3], double sign) {
  double v = 0.0;
  for (int k = 0; k < 3; ++k) {
    const bool hi = (n[k] * sign) > 0.0;
    v += n[k] * ((hi ? b.hi[k] : b.lo[k]) - o[k]);
  }
  return v;
}

// Conservative float box coordinates: pad by a small multiple of the scene
// scale and of the coordinate, then round outward, so that float slab tests
// on the GPU never cut off a part of the box that holds a triangle.
float pad_down(double v, double scale) {
  const double p = v - (1e-5 * scale + 4e-7 * std::fabs(v));
  float f = (float)p;
  if ((double)f > p) f = std::nextafter(f, -INFINITY);
  return f;
}
float pad_up(double v, double scale) {
  const double p = v + (1e-5 * scale + 4e-7 * std::fabs(v));
  float f = (float)p;
  if ((double)f < p) f = std::nextafter(f, INFINITY);
  return f;
}

struct BNode {       // binary build node
  Box box;
  int32_t left = -1, right = -1;  // children (build indices) for inner nodes
  uint32_t first = 0, count = 0;  // leaf range in the leaf-order reference list
  uint32_t depth = 0;
};

constexpr int kBins = 16;           // object-split bins per axis
constexpr int kSpatialBins = 8;     // spatial-split bins per axis
static_assert(kSpatialBins <= 32, "add_parts keeps at most 32 parts");
constexpr double kCostNode = 1.0;
constexpr double kCostTri = 1.2;
// Spatial splits are tried where the best object split's children overlap by
// more than this share of the root's surface area.  A smaller share spends the
// reference budget near the fan centres at the top of the tree; on the
// 4,096-triangle cylinder 1e-3 halves the triangle tests per particle, where
// 1e-5 removes a quarter.
constexpr double kSpatialAlpha = 1e-3;
constexpr double kRefBudget = 0.5;      // at most this many extra references per triangle, in total
constexpr uint32_t kMaxDepth = kMaxStack - 20;  // SAH below this depth, median splits after
// A side is exposed when no vertex of the mesh lies more than this (m) in front
// of its plane.  The kernel skips a re-emitted ray only when it leaves at more
// than 0.01 from the plane in cos, so a hit it could miss would lie within
// 1e-10 m, below the shortest hit distance the traversal accepts.
constexpr double kExposedEps = 1e-12;

// Corner (bit 0: +x, bit 1: +y, bit 2: +z) that slot s of a W-wide node faces.
uint32_t slot_corner(uint32_t W, uint32_t s) { return W == 8 ? s : kWide4Corner[s]; }

// Lays the binary tree out as compressed W-wide nodes (W = 4 or 8; the
// format is described with kWideLeafMax in tpmc_internal.h).  Returns false,
// leaving `out` untouched, when the wide tree would be deeper than the
// traversal stack; the caller then keeps the binary layout.
bool layout_wide(std::vector<BNode>& bn, const std::vector<uint32_t>& leaf_refs, const std::vector<Prim>& prims,
                 const double* xyz, const uint32_t* tri, uint32_t W, double scale, BvhBuild* out) {
  // 1. leaves of at most kWideLeafMax references: a larger leaf becomes a
  //    binary subtree of leaves with the same box
  for (size_t i = 0; i < bn.size(); ++i) {
    if (bn[i].left >= 0 || bn[i].count <= (uint32_t)kWideLeafMax) continue;
    const uint32_t n = bn[i].count;
    const uint32_t leaves = (n + kWideLeafMax - 1) / kWideLeafMax;
    const uint32_t h = ((leaves + 1) / 2) * kWideLeafMax;  // whole leaves in the first half
    BNode a, b;
    a.box = b.box = bn[i].box;
    a.depth = b.depth = bn[i].depth + 1;
    a.first = bn[i].first;
    a.count = h;
    b.first = a.first + h;
    b.count = n - h;
    const int32_t ia = (int32_t)bn.size();
    bn.push_back(a);
    bn.push_back(b);
    bn[i].left = ia;
    bn[i].right = ia + 1;
    bn[i].count = 0;
  }

  // 2. collapse by the surface-area heuristic (the dynamic programme of
  //    Ylitie, Karras & Laine, restated): every binary node m can fill one
  //    slot of its wide parent, as a leaf (when its subtree holds at most
  //    kWideLeafMax references: the builder emits leaves depth first, so those
  //    form one range of leaf_refs) or as a wide node of its own; or it can be
  //    opened into its two children's slots.  With A the surface area,
  //      leaf(m)  = A(m) c_tri refs(m),   node(m) = A(m) c_node + F(m, W),
  //      slot(m)  = min(leaf(m), node(m)),
  //      G(m, j)  = cheapest way to cover m's subtree with at most j slots
  //               = min(slot(m), F(m, j)) for j >= 2, slot(m) for j = 1,
  //      F(m, j)  = min over j1 + j2 = j of G(left, j1) + G(right, j2).
  //    A triangle cut by a spatial split may then appear twice in one merged
  //    leaf, which only repeats a test.
  constexpr double kWideCostNode = 1.0, kWideCostTri = 0.3;
  constexpr double kInf = INFINITY;
  const size_t nb = bn.size();
  std::vector<uint32_t> sub_refs(nb, 0), sub_first(nb, 0);
  std::vector<double> leaf_cost(nb, kInf), node_cost(nb, kInf), Fc(nb * 9, kInf), Gc(nb * 9, kInf);
  std::vector<int8_t> Fsplit(nb * 9, 0), Gopen(nb * 9, 0);
  for (size_t i = nb; i-- > 0;) {  // children come after their parents in bn
    const BNode& b = bn[i];
    const double A = std::max(b.box.area(), 1e-300);
    if (b.left < 0) {
      sub_refs[i] = b.count;
      sub_first[i] = b.first;
    } else {
      const int32_t l = b.left, r = b.right;
      sub_refs[i] = sub_refs[l] + sub_refs[r];
      sub_first[i] = std::min(sub_first[l], sub_first[r]);
      for (uint32_t j = 2; j <= W; ++j)
        for (uint32_t j1 = 1; j1 < j; ++j1) {
          const double c = Gc[9 * l + j1] + Gc[9 * r + (j - j1)];
          if (c < Fc[9 * i + j]) { Fc[9 * i + j] = c; Fsplit[9 * i + j] = (int8_t)j1; }
        }
      node_cost[i] = A * kWideCostNode + Fc[9 * i + W];
    }
    if (sub_refs[i] <= (uint32_t)kWideLeafMax) leaf_cost[i] = A * kWideCostTri * sub_refs[i];
    const double slot = std::min(leaf_cost[i], node_cost[i]);
    for (uint32_t j = 1; j <= W; ++j) {
      Gc[9 * i + j] = slot;
      if (j >= 2 && Fc[9 * i + j] < slot) { Gc[9 * i + j] = Fc[9 * i + j]; Gopen[9 * i + j] = 1; }
      if (j >= 2 && Gc[9 * i + j - 1] < Gc[9 * i + j]) {  // at most j slots
        Gc[9 * i + j] = Gc[9 * i + j - 1];
        Gopen[9 * i + j] = Gopen[9 * i + j - 1];
        if (Gopen[9 * i + j]) { Fc[9 * i + j] = Fc[9 * i + j - 1]; Fsplit[9 * i + j] = Fsplit[9 * i + j - 1]; }
      }
    }
  }
  // the binary nodes that fill the slots of the wide node made from binary node m
  std::vector<int32_t> cover;
  auto collect = [&](auto&& self, int32_t m, uint32_t j) -> void {
    if (Gopen[9 * m + j]) {
      const uint32_t j1 = (uint32_t)Fsplit[9 * m + j];
      self(self, bn[m].left, j1);
      self(self, bn[m].right, j - j1);
    } else {
      cover.push_back(m);
    }
  };
  auto is_leaf_slot = [&](int32_t m) { return leaf_cost[m] <= node_cost[m]; };

  //    The children go to the slots whose corners point most nearly from the
  //    node's centre to theirs (greedy over all child-slot pairs), and the
  //    inner ones get consecutive wide indices in slot order.
  struct WideNode {
    int32_t b;                  // binary node
    int32_t kid[8];             // binary node in each slot, or -1
    uint32_t depth;
  };
  std::vector<WideNode> wn;
  wn.push_back(WideNode{0, {-1, -1, -1, -1, -1, -1, -1, -1}, 1});
  uint32_t max_depth = 1;
  std::vector<char> leaf_slot(nb, 0);
  for (size_t w = 0; w < wn.size(); ++w) {
    cover.clear();
    const int32_t b0i = wn[w].b;
    if (bn[b0i].left < 0) {
      cover.push_back(b0i);  // a tree that is a single leaf
    } else {
      const uint32_t j1 = (uint32_t)Fsplit[9 * b0i + W];
      collect(collect, bn[b0i].left, j1);
      collect(collect, bn[b0i].right, W - j1);
    }
    const std::vector<int32_t> kids(cover);
    for (int32_t k : kids) leaf_slot[k] = (bn[k].left < 0 || is_leaf_slot(k)) ? 1 : 0;
    const BNode& b0 = bn[b0i];
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = 0.5 * (b0.box.lo[a] + b0.box.hi[a]);
    struct Pair { double score; uint32_t k, s; };
    std::vector<Pair> pairs;
    for (uint32_t k = 0; k < kids.size(); ++k)
      for (uint32_t s = 0; s < W; ++s) {
        const uint32_t corner = slot_corner(W, s);
        const Box& kb = bn[kids[k]].box;
        double score = 0.0;
        for (int a = 0; a < 3; ++a) score += (0.5 * (kb.lo[a] + kb.hi[a]) - c[a]) * (((corner >> a) & 1u) ? 1.0 : -1.0);
        pairs.push_back(Pair{score, k, s});
      }
    std::stable_sort(pairs.begin(), pairs.end(), [](const Pair& x, const Pair& y) { return x.score > y.score; });
    std::vector<char> kid_done(kids.size(), 0), slot_done(W, 0);
    for (const Pair& pr : pairs) {
      if (kid_done[pr.k] || slot_done[pr.s]) continue;
      kid_done[pr.k] = slot_done[pr.s] = 1;
      wn[w].kid[pr.s] = kids[pr.k];
    }
    for (uint32_t s = 0; s < W; ++s) {
      const int32_t k = wn[w].kid[s];
      if (k >= 0 && !leaf_slot[k]) {
        wn.push_back(WideNode{k, {-1, -1, -1, -1, -1, -1, -1, -1}, wn[w].depth + 1});
        max_depth = std::max(max_depth, wn[w].depth + 1);
      }
    }
  }
  // the traversal stack holds one group per level; child indices take 24 bits
  if (max_depth + 1 >= (uint32_t)kMaxStackW || wn.size() >= (1u << 24)) return false;

  // 3. nodes and the triangle blocks, in wide-node order
  const uint32_t F4 = W == 8 ? 5 : 4;
  size_t n_refs = 0;
  for (const WideNode& x : wn)
    for (uint32_t s = 0; s < W; ++s)
      if (x.kid[s] >= 0 && leaf_slot[x.kid[s]]) n_refs += sub_refs[x.kid[s]];
  float* nodes = (float*)std::calloc(wn.size() * F4 * 4, sizeof(float));
  float* tris = (float*)std::calloc(std::max<size_t>(n_refs, 1) * 12, sizeof(float));
  double* tris64 = (double*)std::calloc(std::max<size_t>(n_refs, 1) * 12, sizeof(double));
  uint32_t next_inner = 1, leaf_max = 0;
  size_t ref = 0;
  for (size_t w = 0; w < wn.size(); ++w) {
    uint32_t* nd = reinterpret_cast<uint32_t*>(nodes + w * F4 * 4);
    float lo[8][3], hi[8][3];
    double p[3], top[3];
    for (int a = 0; a < 3; ++a) { p[a] = INFINITY; top[a] = -INFINITY; }
    for (uint32_t s = 0; s < W; ++s) {
      const int32_t k = wn[w].kid[s];
      if (k < 0) continue;
      for (int a = 0; a < 3; ++a) {
        lo[s][a] = pad_down(bn[k].box.lo[a], scale);
        hi[s][a] = pad_up(bn[k].box.hi[a], scale);
        p[a] = std::min(p[a], (double)lo[s][a]);
        top[a] = std::max(top[a], (double)hi[s][a]);
      }
    }
    // grid: origin p (a float), step 2^e_a with (top - p) <= 255 2^e_a
    int e[3];
    for (int a = 0; a < 3; ++a) {
      const double ext = top[a] - p[a];
      int ea = ext > 0.0 ? (int)std::ceil(std::log2(ext / 255.0)) : -126;
      ea = std::min(std::max(ea, -126), 127);
      while (ea < 127 && ext > 255.0 * std::ldexp(1.0, ea)) ++ea;
      while (ea > -126 && ext <= 255.0 * std::ldexp(1.0, ea - 1)) --ea;
      e[a] = ea;
      const float pf = (float)p[a];  // exact: p is the smallest of the children's float corners
      std::memcpy(&nd[a], &pf, 4);
    }
    uint32_t imask = 0;
    for (uint32_t s = 0; s < W; ++s)
      if (wn[w].kid[s] >= 0 && !leaf_slot[wn[w].kid[s]]) imask |= 1u << s;
    nd[3] = (uint32_t)(e[0] + 127) | ((uint32_t)(e[1] + 127) << 8) | ((uint32_t)(e[2] + 127) << 16) | (imask << 24);
    nd[4] = imask ? next_inner : 0u;
    nd[5] = (uint32_t)ref;
    for (uint32_t s = 0; s < W; ++s)
      if ((imask >> s) & 1u) ++next_inner;
    // quantised planes (empty slots: lo 255 > hi 0) and leaf metadata
    auto put = [&](uint32_t word, uint32_t byte, uint32_t v) { nd[word] = (nd[word] & ~(0xFFu << (8 * byte))) | (v << (8 * byte)); };
    const uint32_t per_plane = W == 8 ? 2 : 1;
    for (uint32_t s = 0; s < W; ++s) {
      const int32_t k = wn[w].kid[s];
      for (int plane = 0; plane < 6; ++plane) {
        const int a = plane % 3;
        uint32_t q = plane < 3 ? 255u : 0u;
        if (k >= 0) {
          const double step = std::ldexp(1.0, e[a]);
          const double v = plane < 3 ? std::floor(((double)lo[s][a] - p[a]) / step)
                                     : std::ceil(((double)hi[s][a] - p[a]) / step);
          q = (uint32_t)std::min(255.0, std::max(0.0, v));
        }
        put(8 + per_plane * plane + s / 4, s % 4, q);
      }
      if (k >= 0 && leaf_slot[k]) {
        const uint32_t count = sub_refs[k], first = sub_first[k];
        const uint32_t off = (uint32_t)(ref - nd[5]);
        put(6 + s / 4, s % 4, ((count - 1) << 5) | off);
        leaf_max = std::max(leaf_max, count);
        for (uint32_t j = 0; j < count; ++j, ++ref) {
          const uint32_t id = prims[leaf_refs[first + j]].id;
          for (int v = 0; v < 3; ++v) {
            const double* pv = xyz + 3 * (uint64_t)tri[3 * (size_t)id + v];
            for (int a = 0; a < 3; ++a) {
              tris[12 * ref + 4 * v + a] = (float)pv[a];
              tris64[12 * ref + 3 * v + a] = pv[a];
            }
          }
          std::memcpy(&tris[12 * ref + 3], &id, 4);
          tris64[12 * ref + 9] = (double)id;
        }
      }
    }
  }
  out->nodes = nodes;
  out->tris = tris;
  out->tris64 = tris64;
  out->n_nodes = wn.size();
  out->n_leaf_tris = (uint32_t)n_refs;
  out->width = W;
  out->node_bytes = 16 * F4;
  out->depth = max_depth;
  out->leaf_max = leaf_max;
  return true;
}

}  // namespace

bool build_bvh(const double* xyz, uint32_t n_vert, const uint32_t* tri, uint32_t n_tri, uint32_t max_leaf,
               uint32_t width, BvhBuild* out, const char** err) {
  *out = BvhBuild();
  if (width != 2 && width != 4 && width != 8) { *err = "BVH width must be 2, 4 or 8"; return false; }
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
    p.v[0] = a; p.v[1] = b; p.v[2] = c;
    p.id = i;
    prims.push_back(p);
  }

  // ---- SAH build with spatial splits (iterative, depth first) ----
  std::vector<BNode> bn;
  std::vector<uint32_t> leaf_refs;  // prims index of each reference, in leaf order
  const size_t max_refs =
      std::min<size_t>((size_t)(prims.size() * (1.0 + kRefBudget)) + 1, (size_t)(1u << 24) - 1);
  size_t n_refs = prims.size();
  struct Task {
    int32_t node;
    std::vector<Ref> refs;
  };
  std::vector<Task> todo;
  double root_area = 0.0;
  if (!prims.empty()) {
    Task t;
    t.node = 0;
    t.refs.resize(prims.size());
    BNode root;
    for (uint32_t k = 0; k < prims.size(); ++k) {
      t.refs[k].box = prims[k].box;
      t.refs[k].p = k;
      root.box.grow(prims[k].box);
    }
    root_area = root.box.area();
    bn.push_back(root);
    todo.push_back(std::move(t));
  }
  while (!todo.empty()) {
    Task task = std::move(todo.back());
    todo.pop_back();
    std::vector<Ref>& refs = task.refs;
    const int32_t ni = task.node;
    const BNode nd = bn[ni];
    const uint32_t count = (uint32_t)refs.size();
    const double inv_area = 1.0 / std::max(nd.box.area(), 1e-300);

    // object split: binned SAH over the centroids of the reference boxes
    Box cb;
    for (const Ref& r : refs) {
      double c[3];
      for (int k = 0; k < 3; ++k) c[k] = 0.5 * (r.box.lo[k] + r.box.hi[k]);
      cb.grow(c);
    }
    int obj_axis = -1, obj_bin = -1;
    double obj_cost = INFINITY, obj_overlap = 0.0;
    auto centroid_bin = [&](const Ref& r, int a) {
      const double ext = cb.hi[a] - cb.lo[a];
      int b = (int)((0.5 * (r.box.lo[a] + r.box.hi[a]) - cb.lo[a]) / ext * kBins);
      return std::min(std::max(b, 0), kBins - 1);
    };
    if (count > 1) {
      for (int a = 0; a < 3; ++a) {
        if (!(cb.hi[a] - cb.lo[a] > 0.0)) continue;
        Box bins[kBins];
        uint32_t cnt[kBins] = {0};
        for (const Ref& r : refs) {
          const int b = centroid_bin(r, a);
          bins[b].grow(r.box);
          ++cnt[b];
        }
        Box lbox[kBins], rbox[kBins];
        uint32_t lcnt[kBins], rcnt[kBins];
        Box acc;
        uint32_t c = 0;
        for (int b = 0; b < kBins; ++b) { acc.grow(bins[b]); c += cnt[b]; lbox[b] = acc; lcnt[b] = c; }
        acc = Box();
        c = 0;
        for (int b = kBins - 1; b >= 0; --b) { acc.grow(bins[b]); c += cnt[b]; rbox[b] = acc; rcnt[b] = c; }
        for (int b = 0; b + 1 < kBins; ++b) {
          if (lcnt[b] == 0 || rcnt[b + 1] == 0) continue;
          const double cost =
              kCostNode + kCostTri * (lbox[b].area() * lcnt[b] + rbox[b + 1].area() * rcnt[b + 1]) * inv_area;
          if (cost < obj_cost) {
            obj_cost = cost;
            obj_axis = a;
            obj_bin = b;
            obj_overlap = intersect(lbox[b], rbox[b + 1]).area();
          }
        }
      }
    }

    // spatial split: planes at bin boundaries of the node box; a reference
    // that spans several bins adds the box of its part to each of them
    int sp_axis = -1, sp_bin = -1;
    double sp_cost = INFINITY;
    const bool try_spatial = count > 1 && nd.depth < kMaxDepth && n_refs + count <= max_refs &&
                             obj_overlap > kSpatialAlpha * root_area;
    if (try_spatial) {
      for (int a = 0; a < 3; ++a) {
        const double lo = nd.box.lo[a], ext = nd.box.hi[a] - nd.box.lo[a];
        if (!(ext > 0.0)) continue;
        const double w = ext / kSpatialBins;
        auto bin_of = [&](double x) { return std::min(std::max((int)((x - lo) / w), 0), kSpatialBins - 1); };
        Box bins[kSpatialBins];
        uint32_t enter[kSpatialBins] = {0}, leave[kSpatialBins] = {0};
        for (const Ref& r : refs) {
          const int b0 = bin_of(r.box.lo[a]), b1 = bin_of(r.box.hi[a]);
          ++enter[b0];
          ++leave[b1];
          if (b0 == b1) {
            bins[b0].grow(r.box);
          } else {
            add_parts(prims[r.p], r.box, a, lo, w, b0, b1, bins);
          }
        }
        Box rbox[kSpatialBins];
        uint32_t rcnt[kSpatialBins];
        Box acc;
        uint32_t c = 0;
        for (int b = kSpatialBins - 1; b >= 0; --b) { acc.grow(bins[b]); c += leave[b]; rbox[b] = acc; rcnt[b] = c; }
        acc = Box();
        c = 0;
        for (int b = 0; b + 1 < kSpatialBins; ++b) {
          acc.grow(bins[b]);
          c += enter[b];
          if (c == 0 || rcnt[b + 1] == 0 || (c == count && rcnt[b + 1] == count)) continue;
          const double cost = kCostNode + kCostTri * (acc.area() * c + rbox[b + 1].area() * rcnt[b + 1]) * inv_area;
          if (cost < sp_cost) { sp_cost = cost; sp_axis = a; sp_bin = b; }
        }
      }
    }

    const double leaf_cost = kCostTri * count;
    const bool must_split = count > max_leaf;
    const double best_cost = std::min(obj_cost, sp_cost);
    bool make_leaf = count <= 1 || nd.depth >= kMaxDepth || (!must_split && best_cost >= leaf_cost);
    if (make_leaf && count <= 127) {
      bn[ni].first = (uint32_t)leaf_refs.size();
      bn[ni].count = count;
      for (const Ref& r : refs) leaf_refs.push_back(r.p);
      continue;
    }
    std::vector<Ref> lref, rref;
    bool split_done = false;
    if (!make_leaf && sp_cost < obj_cost) {
      const int a = sp_axis;
      const double lo = nd.box.lo[a], w = (nd.box.hi[a] - nd.box.lo[a]) / kSpatialBins;
      const double plane = lo + (sp_bin + 1) * w;
      auto bin_of = [&](double x) { return std::min(std::max((int)((x - lo) / w), 0), kSpatialBins - 1); };
      for (const Ref& r : refs) {
        const int b0 = bin_of(r.box.lo[a]), b1 = bin_of(r.box.hi[a]);
        if (b1 <= sp_bin) {
          lref.push_back(r);
        } else if (b0 > sp_bin) {
          rref.push_back(r);
        } else {
          Ref l = r, rr = r;
          split_ref(prims[r.p], r.box, a, plane, l.box, rr.box);
          if (l.box.empty() && rr.box.empty()) {
            // rounding left neither side a box: keep the whole part on both
            l.box = r.box;
            rr.box = r.box;
          }
          if (!l.box.empty()) lref.push_back(l);
          if (!rr.box.empty()) rref.push_back(rr);
        }
      }
      split_done = !lref.empty() && !rref.empty() && (lref.size() < count || rref.size() < count);
      if (split_done) n_refs += lref.size() + rref.size() - count;
      else { lref.clear(); rref.clear(); }
    }
    if (!split_done) {
      if (!make_leaf && obj_axis >= 0) {
        for (const Ref& r : refs) (centroid_bin(r, obj_axis) <= obj_bin ? lref : rref).push_back(r);
      }
      if (lref.empty() || rref.empty()) {
        // all centroids coincide, no useful bin, or an oversized leaf at the
        // depth limit: split the list in half
        lref.assign(refs.begin(), refs.begin() + count / 2);
        rref.assign(refs.begin() + count / 2, refs.end());
      }
    }
    std::vector<Ref>().swap(refs);
    BNode l, r;
    l.depth = r.depth = nd.depth + 1;
    for (const Ref& x : lref) l.box.grow(x.box);
    for (const Ref& x : rref) r.box.grow(x.box);
    const int32_t li = (int32_t)bn.size();
    bn.push_back(l);
    const int32_t ri = (int32_t)bn.size();
    bn.push_back(r);
    bn[ni].left = li;
    bn[ni].right = ri;
    todo.push_back(Task{ri, std::move(rref)});
    todo.push_back(Task{li, std::move(lref)});
  }

  // ---- exposed sides: bit 0 front (the side n points to), bit 1 back ----
  // Branch and bound over the build tree: a node whose box lies wholly behind
  // the plane holds no vertex in front of it.  Every vertex lies in the box of
  // some leaf that references its triangle, so pruning is exact.
  if (!bn.empty()) {
    // The vertices that reach farthest along 26 directions (axes, face and
    // space diagonals): most sides that are not exposed see one of them in
    // front, which settles them without a search.
    std::vector<const double*> probes;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          const double* best = nullptr;
          double bv = -INFINITY;
          for (const Prim& t : prims)
            for (int j = 0; j < 3; ++j) {
              const double* v = t.v[j];
              const double h = dx * v[0] + dy * v[1] + dz * v[2];
              if (h > bv) { bv = h; best = v; }
            }
          if (best) probes.push_back(best);
        }
    auto side_clear = [&](const Prim& t, const double n[3], double sign, std::vector<int32_t>& stack) {
      const double* o = t.v[0];
      for (const double* v : probes)
        if (sign * (n[0] * (v[0] - o[0]) + n[1] * (v[1] - o[1]) + n[2] * (v[2] - o[2])) > kExposedEps) return false;
      stack.assign(1, 0);
      while (!stack.empty()) {
        const BNode& nd = bn[stack.back()];
        stack.pop_back();
        if (sign * box_extreme(nd.box, n, o, sign) <= kExposedEps) continue;
        if (nd.left >= 0) {
          // the child reaching farther in front is searched first
          const bool l_first = sign * box_extreme(bn[nd.left].box, n, o, sign) >=
                               sign * box_extreme(bn[nd.right].box, n, o, sign);
          stack.push_back(l_first ? nd.right : nd.left);
          stack.push_back(l_first ? nd.left : nd.right);
          continue;
        }
        for (uint32_t k = nd.first; k < nd.first + nd.count; ++k)
          for (int j = 0; j < 3; ++j) {
            const double* v = prims[leaf_refs[k]].v[j];
            const double h = n[0] * (v[0] - o[0]) + n[1] * (v[1] - o[1]) + n[2] * (v[2] - o[2]);
            if (sign * h > kExposedEps) return false;
          }
      }
      return true;
    };
    auto work = [&](size_t begin, size_t end) {
      std::vector<int32_t> stack;
      for (size_t k = begin; k < end; ++k) {
        const Prim& t = prims[k];
        const double* f = out->frames64 + 8 * (size_t)t.id;
        const double n[3] = {f[0], f[1], f[2]};
        uint32_t bits = 0;
        if (side_clear(t, n, 1.0, stack)) bits |= 1u;
        if (side_clear(t, n, -1.0, stack)) bits |= 2u;
        out->frames64[8 * (size_t)t.id + 7] = (double)bits;
        std::memcpy(out->frames + 8 * (size_t)t.id + 7, &bits, 4);
      }
    };
    const size_t n_prims = prims.size();
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const size_t n_threads = n_prims < 1024 ? 1 : std::min<size_t>(hw, n_prims / 512);
    if (n_threads <= 1) {
      work(0, n_prims);
    } else {
      std::vector<std::thread> th;
      for (size_t w = 0; w < n_threads; ++w)
        th.emplace_back(work, n_prims * w / n_threads, n_prims * (w + 1) / n_threads);
      for (auto& t : th) t.join();
    }
    for (const Prim& t : prims) {
      const uint32_t bits = (uint32_t)out->frames64[8 * (size_t)t.id + 7];
      out->n_exposed += (bits & 1u) + ((bits >> 1) & 1u);
    }
  }

  if (!bn.empty())
    for (int a = 0; a < 3; ++a) {
      out->root_lo[a] = pad_down(bn[0].box.lo[a], scale);
      out->root_hi[a] = pad_up(bn[0].box.hi[a], scale);
    }
  out->width = 2;
  out->node_bytes = 64;
  if (width > 2 && !bn.empty() && layout_wide(bn, leaf_refs, prims, xyz, tri, width, scale, out)) return true;

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
  out->node_bytes = 32;
  out->nodes = (float*)std::calloc(std::max<size_t>(n_nodes, 1) * 8, sizeof(float));

  // triangles in leaf order
  out->n_leaf_tris = (uint32_t)leaf_refs.size();
  out->tris = (float*)std::calloc(std::max<size_t>(leaf_refs.size(), 1) * 12, sizeof(float));
  out->tris64 = (double*)std::calloc(std::max<size_t>(leaf_refs.size(), 1) * 12, sizeof(double));
  for (size_t k = 0; k < leaf_refs.size(); ++k) {
    const uint32_t i = prims[leaf_refs[k]].id;
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

  // The boxes' grid: a step 2^e per axis with the padded root box inside
  // 65,533 steps, and an origin one step below it, so that every box,
  // widened by one step each way, keeps its coordinates in [0, 65535].
  for (int a = 0; a < 3 && !bn.empty(); ++a) {
    const double ext = std::max((double)out->root_hi[a] - (double)out->root_lo[a], 1e-30);
    int e = (int)std::ceil(std::log2(ext / 65533.0));
    while (std::ldexp(65533.0, e) < ext) ++e;
    const double step = std::ldexp(1.0, e);
    float origin = (float)((double)out->root_lo[a] - step);
    if ((double)origin > (double)out->root_lo[a] - step) origin = std::nextafter(origin, -INFINITY);
    out->qorigin[a] = origin;
    out->qstep[a] = (float)step;
  }
  auto qcoord = [&](double v, int a, bool up) {
    const double x = (v - (double)out->qorigin[a]) / (double)out->qstep[a];
    const double q = up ? std::ceil(x) + 1.0 : std::floor(x) - 1.0;
    return (uint32_t)std::min(65535.0, std::max(0.0, q));
  };
  auto child_code = [&](int32_t b, uint32_t& depth_seen) -> int32_t {
    const BNode& c = bn[b];
    depth_seen = std::max(depth_seen, c.depth);
    if (c.left >= 0) return gpu_index[b];
    out->leaf_max = std::max(out->leaf_max, c.count);
    return ~(int32_t)((c.count << 24) | c.first);
  };
  uint32_t qlo_root[3] = {65535u, 65535u, 65535u}, qhi_root[3] = {0u, 0u, 0u};
  // writes a child's box (null: the empty child, a point at the grid's far
  // corner) into its three words; grows the root's grid box when asked
  auto write_child = [&](uint32_t* nd, int slot, const Box* box, bool root) {
    uint32_t qlo[3], qhi[3];
    for (int a = 0; a < 3; ++a) {
      qlo[a] = box ? qcoord(pad_down(box->lo[a], scale), a, false) : 65535u;
      qhi[a] = box ? qcoord(pad_up(box->hi[a], scale), a, true) : 65535u;
      if (root && box) {
        qlo_root[a] = std::min(qlo_root[a], qlo[a]);
        qhi_root[a] = std::max(qhi_root[a], qhi[a]);
      }
    }
    uint32_t* w = nd + 3 * slot;
    for (int a = 0; a < 3; ++a) w[a] = qlo[a] | (qhi[a] << 16);
  };
  uint32_t depth_seen = 0;
  uint32_t* nodes = reinterpret_cast<uint32_t*>(out->nodes);
  if (single_leaf) {
    write_child(nodes, 0, &bn[0].box, true);
    write_child(nodes, 1, nullptr, true);
    int32_t c0 = child_code(0, depth_seen), c1 = ~(int32_t)0;  // empty leaf: count 0
    std::memcpy(nodes + 6, &c0, 4);
    std::memcpy(nodes + 7, &c1, 4);
  } else {
    for (size_t g = 0; g < inner_order.size(); ++g) {
      const BNode& b = bn[inner_order[g]];
      uint32_t* nd = nodes + 8 * g;
      write_child(nd, 0, &bn[b.left].box, g == 0);
      write_child(nd, 1, &bn[b.right].box, g == 0);
      int32_t c0 = child_code(b.left, depth_seen), c1 = child_code(b.right, depth_seen);
      std::memcpy(nd + 6, &c0, 4);
      std::memcpy(nd + 7, &c1, 4);
    }
  }
  // the root box in the grid units the kernel's slab test reads: 2^23 + q
  for (int a = 0; a < 3 && n_nodes > 0; ++a) {
    out->qroot_lo[a] = 8388608.0f + (float)qlo_root[a];
    out->qroot_hi[a] = 8388608.0f + (float)qhi_root[a];
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
