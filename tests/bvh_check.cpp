// Host check of the BVH builder (paper_1312_3691_gb300/csrc/bvh.cpp).
//
// Builds the hierarchy exactly as tpmc_mesh_load does, then, for every ray of
// a ray file, finds the closest hit twice with one and the same double
// precision ray/triangle test: by walking the built tree (the float boxes
// as laid out for the GPU, culled against the best hit so far, inclusive)
// and by brute force over all triangles.  Nearest t wins; equal t goes to the
// lower triangle index.  A tree that loses any part of a triangle (a spatial
// split that drops a piece, a box that does not contain its part) shows up as
// a ray whose two answers differ.  Also checks that every triangle with
// nonzero area is referenced by some leaf, that leaves respect the size
// limit (more than max_leaf only where the depth limit stops the build, and
// never more than 127), and that every triangle side marked exposed has the
// whole mesh behind its plane.
//
// With WIDTH 4 or 8 the tree is laid out as compressed wide nodes, and the
// walk decodes each child box from the node's 8-bit grid exactly as the GPU
// reads it (origin p, step 2^e, bytes qlo / qhi), in double: a quantised box
// that does not contain its child's triangles shows up the same way.
//
// usage: bvh_check MESH RAYS MAX_LEAF [WIDTH]
//   MESH: uint32 n_vert, uint32 n_tri, double xyz[n_vert][3], uint32 tri[n_tri][3]
//   RAYS: uint32 n_rays, double ray[n_rays][6] (origin, direction)
// prints one line: rays mismatches hits n_tri n_refs n_nodes depth leaf_max unreferenced oversized
//                  exposed wrong_exposed width node_bytes bad_index
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "tpmc_internal.h"

namespace {

bool read_all(const char* path, std::vector<unsigned char>& out) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  unsigned char buf[1 << 16];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) out.insert(out.end(), buf, buf + n);
  std::fclose(f);
  return true;
}

// Moller-Trumbore; boundary inclusive.  Returns t or -1.  A determinant below
// 1e-12 of |e1| |e2| |d| (a collinear triangle, or a ray in the triangle's
// plane) counts as no hit: rounding would otherwise turn it into a spurious
// hit far from the triangle.
double hit(const double* o, const double* d, const double* a, const double* b, const double* c) {
  double e1[3], e2[3], s[3];
  for (int i = 0; i < 3; ++i) { e1[i] = b[i] - a[i]; e2[i] = c[i] - a[i]; s[i] = o[i] - a[i]; }
  const double p[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
  const double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
  const double scale = std::sqrt((e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]) *
                                 (e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]) * (d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
  if (!(std::fabs(det) > 1e-12 * scale)) return -1.0;
  const double inv = 1.0 / det;
  const double u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) * inv;
  if (u < 0.0 || u > 1.0) return -1.0;
  const double q[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]};
  const double v = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) * inv;
  if (v < 0.0 || u + v > 1.0) return -1.0;
  const double t = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) * inv;
  return t > 1e-12 ? t : -1.0;
}

struct Best {
  double t = INFINITY;
  uint32_t id = 0xFFFFFFFFu;
  void offer(double t2, uint32_t id2) {
    if (t2 < 0.0) return;
    if (t2 < t || (t2 == t && id2 < id)) { t = t2; id = id2; }
  }
};

}  // namespace

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  std::vector<unsigned char> mb, rb;
  if (!read_all(argv[1], mb) || !read_all(argv[2], rb)) return 3;
  const uint32_t max_leaf = (uint32_t)std::atoi(argv[3]);
  const uint32_t width = argc > 4 ? (uint32_t)std::atoi(argv[4]) : 2u;
  uint32_t nv, nt, nr;
  std::memcpy(&nv, mb.data(), 4);
  std::memcpy(&nt, mb.data() + 4, 4);
  std::vector<double> xyz(3 * (size_t)nv);
  std::vector<uint32_t> tri(3 * (size_t)nt);
  std::memcpy(xyz.data(), mb.data() + 8, xyz.size() * 8);
  std::memcpy(tri.data(), mb.data() + 8 + xyz.size() * 8, tri.size() * 4);
  std::memcpy(&nr, rb.data(), 4);
  std::vector<double> rays(6 * (size_t)nr);
  std::memcpy(rays.data(), rb.data() + 4, rays.size() * 8);

  tpmc::BvhBuild b;
  const char* err = nullptr;
  if (!tpmc::build_bvh(xyz.data(), nv, tri.data(), nt, max_leaf, width, &b, &err)) {
    std::printf("build failed: %s\n", err ? err : "?");
    return 4;
  }
  auto vert = [&](uint32_t t, int k) { return xyz.data() + 3 * (size_t)tri[3 * (size_t)t + k]; };

  // references: every triangle with nonzero area appears in some leaf
  std::vector<char> seen(nt, 0);
  for (uint32_t k = 0; k < b.n_leaf_tris; ++k) {
    uint32_t id;
    std::memcpy(&id, b.tris + 12 * (size_t)k + 3, 4);
    if (id < nt) seen[id] = 1;
  }
  uint32_t unreferenced = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    const double* a = vert(t, 0);
    const double* bb = vert(t, 1);
    const double* c = vert(t, 2);
    const double e1[3] = {bb[0] - a[0], bb[1] - a[1], bb[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const bool nonzero = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) > 0.0;
    if (nonzero && !seen[t]) ++unreferenced;
  }

  // leaves within the size limit
  uint32_t oversized = 0;
  std::vector<int32_t> stack;
  for (size_t g = 0; g < b.n_nodes && b.width == 2; ++g)
    for (int c = 0; c < 2; ++c) {
      int32_t code;
      std::memcpy(&code, b.nodes + 8 * g + 6 + c, 4);
      if (code < 0 && ((~(uint32_t)code) >> 24) > 127u) ++oversized;
    }

  // exposed sides: a side marked in the frame's word 7 has no vertex more
  // than 1e-12 m in front of its plane (brute force over all vertices)
  uint32_t exposed = 0, wrong_exposed = 0;
  for (uint32_t t = 0; t < nt; ++t) {
    const double* f = b.frames64 + 8 * (size_t)t;
    const uint32_t bits = (uint32_t)f[7];
    uint32_t fbits;
    std::memcpy(&fbits, b.frames + 8 * (size_t)t + 7, 4);
    if (fbits != bits) ++wrong_exposed;
    const double* a = vert(t, 0);
    for (int side = 0; side < 2; ++side) {
      if (!((bits >> side) & 1u)) continue;
      ++exposed;
      const double sg = side == 0 ? 1.0 : -1.0;
      for (uint32_t v = 0; v < nv; ++v) {
        const double* p = xyz.data() + 3 * (size_t)v;
        if (sg * (f[0] * (p[0] - a[0]) + f[1] * (p[1] - a[1]) + f[2] * (p[2] - a[2])) > 1e-12) { ++wrong_exposed; break; }
      }
    }
  }

  uint64_t mismatches = 0, hits = 0, bad_index = 0;  // bad_index: a child or triangle outside its array
  for (uint32_t r = 0; r < nr; ++r) {
    const double* o = rays.data() + 6 * (size_t)r;
    const double* d = o + 3;
    Best brute;
    for (uint32_t t = 0; t < nt; ++t) brute.offer(hit(o, d, vert(t, 0), vert(t, 1), vert(t, 2)), t);
    Best walk;
    auto slab = [&](const double lo[3], const double hi[3]) {
      double tn = 0.0, tf = walk.t;
      for (int i = 0; i < 3; ++i) {
        if (d[i] == 0.0) {
          if (o[i] < lo[i] || o[i] > hi[i]) tn = INFINITY;
          continue;
        }
        const double t0 = (lo[i] - o[i]) / d[i], t1 = (hi[i] - o[i]) / d[i];
        tn = std::fmax(tn, std::fmin(t0, t1));
        tf = std::fmin(tf, std::fmax(t0, t1));
      }
      return tn <= tf;
    };
    if (b.n_nodes > 0 && b.width > 2) {
      const uint32_t W = b.width, F = b.node_bytes / 4, per_plane = W == 8 ? 2 : 1;
      stack.assign(1, 0);
      while (!stack.empty()) {
        const uint32_t* nd = reinterpret_cast<const uint32_t*>(b.nodes) + (size_t)F * stack.back();
        stack.pop_back();
        auto byte = [&](uint32_t word, uint32_t k) { return (nd[word] >> (8 * k)) & 0xFFu; };
        float p[3];
        std::memcpy(p, nd, 12);
        const uint32_t imask = nd[3] >> 24;
        for (uint32_t s = 0; s < W; ++s) {
          double lo[3], hi[3];
          bool empty = false;
          for (int a = 0; a < 3; ++a) {
            const double step = std::ldexp(1.0, (int)byte(3, a) - 127);
            const uint32_t ql = byte(8 + per_plane * a + s / 4, s % 4), qh = byte(8 + per_plane * (a + 3) + s / 4, s % 4);
            empty = empty || ql > qh;
            lo[a] = (double)p[a] + step * ql;
            hi[a] = (double)p[a] + step * qh;
          }
          if (empty || !slab(lo, hi)) continue;
          if ((imask >> s) & 1u) {
            const uint32_t child = nd[4] + __builtin_popcount(imask & ((1u << s) - 1u));
            if (child >= b.n_nodes || child == 0) { ++bad_index; continue; }
            stack.push_back((int32_t)child);
          } else {
            const uint32_t meta = byte(6 + s / 4, s % 4), first = nd[5] + (meta & 31u), count = (meta >> 5) + 1;
            if ((meta & 31u) + count > 32u || first + count > b.n_leaf_tris) { ++bad_index; continue; }
            for (uint32_t k = first; k < first + count; ++k) {
              uint32_t id;
              std::memcpy(&id, b.tris + 12 * (size_t)k + 3, 4);
              walk.offer(hit(o, d, vert(id, 0), vert(id, 1), vert(id, 2)), id);
            }
          }
        }
      }
    } else if (b.n_nodes > 0) {
      // binary nodes: 16-bit boxes on the mesh's grid, decoded exactly in double
      stack.assign(1, 0);
      while (!stack.empty()) {
        const int32_t node = stack.back();
        stack.pop_back();
        if (node < 0 || (size_t)node >= b.n_nodes) { ++bad_index; continue; }
        const uint32_t* nd = reinterpret_cast<const uint32_t*>(b.nodes) + 8 * (size_t)node;
        for (int c = 0; c < 2; ++c) {
          const uint32_t* w = nd + 3 * c;
          const uint32_t ql[3] = {w[0] & 0xFFFFu, w[1] & 0xFFFFu, w[2] & 0xFFFFu};
          const uint32_t qh[3] = {w[0] >> 16, w[1] >> 16, w[2] >> 16};
          double lo[3], hi[3];
          for (int a = 0; a < 3; ++a) {
            lo[a] = (double)b.qorigin[a] + (double)b.qstep[a] * ql[a];
            hi[a] = (double)b.qorigin[a] + (double)b.qstep[a] * qh[a];
          }
          if (!slab(lo, hi)) continue;
          int32_t code;
          std::memcpy(&code, nd + 6 + c, 4);
          if (code >= 0) {
            stack.push_back(code);
          } else {
            const uint32_t u = ~(uint32_t)code, first = u & 0xFFFFFFu, count = u >> 24;
            if (first + count > b.n_leaf_tris) { ++bad_index; continue; }
            for (uint32_t k = first; k < first + count; ++k) {
              uint32_t id;
              std::memcpy(&id, b.tris + 12 * (size_t)k + 3, 4);
              walk.offer(hit(o, d, vert(id, 0), vert(id, 1), vert(id, 2)), id);
            }
          }
        }
      }
    }
    if (brute.id != 0xFFFFFFFFu) ++hits;
    if (brute.id != walk.id || !(brute.t == walk.t || (std::isinf(brute.t) && std::isinf(walk.t)))) ++mismatches;
  }
  std::printf("%u %llu %llu %u %u %zu %u %u %u %u %u %u %u %u %llu\n", nr, (unsigned long long)mismatches,
              (unsigned long long)hits, nt, b.n_leaf_tris, b.n_nodes, b.depth, b.leaf_max, unreferenced, oversized,
              exposed, wrong_exposed, b.width, b.node_bytes, (unsigned long long)bad_index);
  b.release();
  return 0;
}
