// FP64 CPU oracle for the test-particle Monte Carlo (TPMC) hot path of
// Parham & Barba, "Finding the Force -- Consistent Particle Seeding for
// Satellite Aerodynamics" (arXiv 1312.3691).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
// statement of what the GPU library computes.  Only the test suite, the smoke
// check and the benchmark's CPU-baseline leg load it.  It shares no code, no
// header and no constant table with the CUDA library: both sides implement
// Philox4x32-10 from its published definition (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the sampling
// rules from the paper.
//
// Everything is double precision.  Each function names the passage of the
// paper it follows:
//   Eq. 2   drifting Maxwellian (§II.A)
//   Eq. 3   flat plate C_D (Sentman, §II.B.1)          -- see plate_cd_*
//   Eq. 4   convex sphere C_D (Bird, §II.B.2)
//   Eq. 7-10 number flux into a sphere (§III.A.1)
//   Eq. 11  position likelihood g(phi|S) (§III.A.1)
//   Eq. 14a-c velocity component densities (§III.A.2)
//   Eq. 15  Rodrigues rotation to body coordinates (§III.A.3)
//   §II.A   closest-hit ray tracing, diffuse re-emission, momentum sum
//   (ext.)  Cercignani-Lampis-Lord surface model, an alternative to §II.A's
//           Maxwell mix (no passage of the paper uses it)
//   §I, §III.A rectangular control volume with uniform positions on its six
//           faces and per-face counts from the flat-plate flux (the ANGARA
//           scheme the paper replaces), with two velocity laws per face
//
// Readings where the paper is silent or ambiguous (inverse-CDF sampling, the
// frame orientation, the re-emission law, the RNG layout, tie and edge rules)
// are stated where they are used.
//
// Parity status: every function here is pinned by a test in tests/ against a
// closed form, a quadrature, an independent sampler or brute force.  The
// multiple-reflection path is pinned on a concave hemispherical shell by
// Pratt's hyperthermal constant (§II.B.3, Eq. 5), re-derived by a view-factor
// quadrature, and by an exact chord construction for specular walls.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;
constexpr double kBoltzmann = 1.380649e-23;  // J/K (SI exact value)

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al. SC'11): ten rounds of two 32x32->64 products,
// the Weyl key schedule, counter (c0..c3), key (k0,k1).
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    const uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    const uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
    const uint32_t n1 = (uint32_t)prod1;
    const uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
    const uint32_t n3 = (uint32_t)prod0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Word -> uniform on (0,1): the top 23 bits plus one half, times 2^-23, i.e.
// (2k+1) 2^-24 with 2k+1 < 2^24.  It is exactly representable in float as well
// as double, so a float consumer and a double consumer see the same number;
// never 0 and never 1 (range [2^-24, 1 - 2^-24]).
double uniform_from_word(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

// Draw layout (the paper uses "random" draws without naming a generator):
//   key     = (seed low 32 bits, seed high 32 bits)
//   counter = (particle id low, particle id high, stream id, block)
//   block 0 : seeding   -> u_x (position), u_theta, u_vn, u_r (Box-Muller radius)
//             from the top 23 bits of its four words, and u_a (Box-Muller
//             angle) from 23 of the low bits the other four leave unused:
//             bits 0-8 of word 0, 0-8 of word 1 and 0-4 of word 2
//   block 2+b: bounce b -> u_gsi (diffuse or specular), u1, u2, u3 (re-emission)
// (Block 1 is not drawn.)
void draw_words(uint64_t seed, uint32_t stream, uint64_t pid, uint32_t block, uint32_t w[4]) {
  const uint32_t ctr[4] = {(uint32_t)pid, (uint32_t)(pid >> 32), stream, block};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox4x32_10(ctr, key, w);
}

void draw_block(uint64_t seed, uint32_t stream, uint64_t pid, uint32_t block, double u[4]) {
  uint32_t w[4];
  draw_words(seed, stream, pid, block, w);
  for (int i = 0; i < 4; ++i) u[i] = uniform_from_word(w[i]);
}

// The five seeding uniforms of particle pid (see the layout above).
void seed_uniforms(uint64_t seed, uint32_t stream, uint64_t pid, double u[5]) {
  uint32_t w[4];
  draw_words(seed, stream, pid, 0, w);
  for (int i = 0; i < 4; ++i) u[i] = uniform_from_word(w[i]);
  const uint32_t low = (w[0] & 0x1FFu) | ((w[1] & 0x1FFu) << 9) | ((w[2] & 0x1Fu) << 18);
  u[4] = uniform_from_word(low << 9);
}

// ---------------------------------------------------------------------------
// Small vector helpers.
// ---------------------------------------------------------------------------
struct V3 {
  double x, y, z;
};
V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double norm(V3 a) { return std::sqrt(dot(a, a)); }
V3 unit(V3 a) { return (1.0 / norm(a)) * a; }
V3 load3(const double* p) { return {p[0], p[1], p[2]}; }
void store3(double* p, V3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }

// ---------------------------------------------------------------------------
// Kinetic-theory closed forms.
// ---------------------------------------------------------------------------

// Eq. 10: Gamma / (c_mp n r^2) = sqrt(pi) e^{-S^2} + (pi/(2S) + pi S) erf S.
double gamma_coefficient(double S) {
  return kSqrtPi * std::exp(-S * S) + (kPi / (2.0 * S) + kPi * S) * std::erf(S);
}

// Eq. 11 denominator: D(S) = e^{-S^2} + sqrt(pi) (1 + 2 S^2) erf(S) / (2 S).
double position_norm(double S) {
  return std::exp(-S * S) + kSqrtPi * (1.0 + 2.0 * S * S) * std::erf(S) / (2.0 * S);
}

// Eq. 11: g(phi|S), the likelihood of the incidence latitude phi in [-pi/2, pi/2].
double g_phi(double phi, double S) {
  const double sp = std::sin(phi);
  return std::cos(phi) * (std::exp(-S * S * sp * sp) + S * kSqrtPi * sp * (1.0 + std::erf(S * sp))) /
         position_norm(S);
}

// The same law in x = sin(phi) (g dphi = h dx, since dx = cos(phi) dphi).
double h_x(double x, double S) {
  return (std::exp(-S * S * x * x) + S * kSqrtPi * x * (1.0 + std::erf(S * x))) / position_norm(S);
}

// Antiderivative of D*h: A(y) = sqrt(pi)/(4S) (2 S^2 y^2 + 1) erf(S y) + sqrt(pi) S y^2 / 2
//                               + (y/2) e^{-S^2 y^2}.
// (d/dy of each term: the erf term gives sqrt(pi) S y erf(Sy) + (1/2 + S^2 y^2) e^{-S^2y^2}
//  ... summing to e^{-S^2 y^2} + sqrt(pi) S y (1 + erf(S y)).)
double position_antiderivative(double y, double S) {
  return kSqrtPi / (4.0 * S) * (2.0 * S * S * y * y + 1.0) * std::erf(S * y) + kSqrtPi * S * y * y / 2.0 +
         0.5 * y * std::exp(-S * S * y * y);
}

// CDF of x = sin(phi): H(x) = [A(x) - A(-1)] / D(S).
double position_cdf(double x, double S) {
  return (position_antiderivative(x, S) - position_antiderivative(-1.0, S)) / position_norm(S);
}

// Monotone root of cdf(x) = u on [lo, hi] by plain bisection until the bracket
// stops shrinking in double precision (the reading of "sample from the
// density": inverse transform with one uniform per coordinate).
template <class F>
double bisect_cdf(F cdf, double u, double lo, double hi) {
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (cdf(mid) < u) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

double position_inverse(double u, double S) {
  return bisect_cdf([S](double x) { return position_cdf(x, S); }, u, -1.0, 1.0);
}

// Eq. 14a with the numerator read as 2 (v_n / c_mp): the density of the inward
// normal speed x = v_n / c_mp > 0 for the normal speed ratio s = S sin(phi):
//   p(x) = 2 x exp(-(x - s)^2) / Z(s),  Z(s) = e^{-s^2} + sqrt(pi) s (1 + erf s).
// 1 + erf(s) is written erfc(-s) so that negative s keeps its digits.
double normal_speed_norm(double s) { return std::exp(-s * s) + kSqrtPi * s * std::erfc(-s); }

double normal_speed_pdf(double x, double s) {
  return x <= 0.0 ? 0.0 : 2.0 * x * std::exp(-(x - s) * (x - s)) / normal_speed_norm(s);
}

// CDF: F(x) = [e^{-s^2} - e^{-(x-s)^2} + sqrt(pi) s (erf(x-s) + erf s)] / Z(s),
// with erf(x-s) + erf(s) = erfc(-s) - erfc(x-s).
double normal_speed_cdf(double x, double s) {
  if (x <= 0.0) return 0.0;
  return (std::exp(-s * s) - std::exp(-(x - s) * (x - s)) + kSqrtPi * s * (std::erfc(-s) - std::erfc(x - s))) /
         normal_speed_norm(s);
}

// Survival function 1 - F(x) = [e^{-(x-s)^2} + sqrt(pi) s erfc(x-s)] / Z(s) of the same law.
double normal_speed_survival(double x, double s) {
  if (x <= 0.0) return 1.0;
  return (std::exp(-(x - s) * (x - s)) + kSqrtPi * s * std::erfc(x - s)) / normal_speed_norm(s);
}

// Inverse transform F(x) = u.  Above the median F rounds to 1 in double
// before the root is resolved, so there the same equation is solved as
// 1 - F(x) = 1 - u on the survival function (1 - u is exact for these u).
double normal_speed_inverse(double u, double s) {
  const double hi = std::max(s, 0.0) + 12.0;  // 1 - F(hi) is far below the smallest uniform, 2^-24
  if (u <= 0.5) return bisect_cdf([s](double x) { return normal_speed_cdf(x, s); }, u, 0.0, hi);
  return bisect_cdf([s](double x) { return -normal_speed_survival(x, s); }, -(1.0 - u), 0.0, hi);
}

// Normal speed of the rectangular-CV seeder's second velocity law: the
// free-stream Maxwellian of Eq. 2 restricted to velocities that enter the face,
// i.e. x = v_n / c_mp > 0 with density exp(-(x - s)^2) / (sqrt(pi)/2 erfc(-s)),
// WITHOUT the flux factor x that Eq. 14a carries.
//   survival Q(x) = erfc(x - s) / erfc(-s),  CDF F(x) = 1 - Q(x).
double truncated_normal_cdf(double x, double s) {
  if (x <= 0.0) return 0.0;
  return (std::erfc(-s) - std::erfc(x - s)) / std::erfc(-s);
}
double truncated_normal_survival(double x, double s) {
  if (x <= 0.0) return 1.0;
  return std::erfc(x - s) / std::erfc(-s);
}
double truncated_normal_inverse(double u, double s) {
  const double hi = std::max(s, 0.0) + 12.0;
  if (u <= 0.5) return bisect_cdf([s](double x) { return truncated_normal_cdf(x, s); }, u, 0.0, hi);
  return bisect_cdf([s](double x) { return -truncated_normal_survival(x, s); }, -(1.0 - u), 0.0, hi);
}

// Per-area fluxes onto a surface element whose inward-normal speed ratio is s
// (free stream of density n, thermal speed c): number flux G, incident normal
// momentum flux P (units n c and n m c^2).  These integrate Eq. 2 over the
// half space of velocities moving into the element.
double flux_G(double s) { return (std::exp(-s * s) + kSqrtPi * s * std::erfc(-s)) / (2.0 * kSqrtPi); }
double flux_P(double s) {
  return (s * std::exp(-s * s) + kSqrtPi * (0.5 + s * s) * std::erfc(-s)) / (2.0 * kSqrtPi);
}

// Force per unit area (units n m c^2) on one side of a surface element with
// outward unit normal nrm, in a free stream of speed ratio S along Vhat,
// without shadowing.  A fraction eps of the molecules is re-emitted diffusely
// at the wall temperature (mean normal speed sqrt(pi)/2 c_W, the flux-weighted
// half-range Maxwellian), the rest specularly.
V3 surface_force(V3 nrm, V3 Vhat, double S, double eps, double cw_over_c) {
  const double vn = dot(Vhat, nrm);
  const double s = -S * vn;  // inward-normal speed ratio
  const V3 tang = S * (Vhat - vn * nrm);  // tangential stream speed ratio (vector)
  const double G = flux_G(s), P = flux_P(s);
  const double normal_push = (2.0 - eps) * P + eps * 0.5 * kSqrtPi * cw_over_c * G;
  return (-normal_push) * nrm + (eps * G) * tang;
}

// ---------------------------------------------------------------------------
// Mesh and closest-hit ray tracing (§II.A: "the closest intersection point to
// the initial position becomes the first collision").
// ---------------------------------------------------------------------------
struct Mesh {
  uint32_t nt = 0;
  std::vector<V3> v0, e1, e2, nrm, t1;
  std::vector<double> area;
  // Median-split bounding-volume hierarchy, used for large meshes only.
  struct Node {
    double lo[3], hi[3];
    int32_t left, right;   // child node indices, -1 for a leaf
    uint32_t first, count;  // leaf range in `order`
  };
  std::vector<Node> nodes;
  std::vector<uint32_t> order;
};

struct Hit {
  bool found = false;
  uint32_t tri = 0;
  double t = 0, u = 0, v = 0;
};

// Moeller & Trumbore (1997) ray/triangle test in double precision.
bool moller_trumbore(const Mesh& m, uint32_t i, V3 o, V3 d, double& t, double& u, double& v) {
  const V3 p = cross(d, m.e2[i]);
  const double det = dot(m.e1[i], p);
  if (det == 0.0 || !std::isfinite(det)) return false;
  const double inv = 1.0 / det;
  const V3 s = o - m.v0[i];
  u = dot(s, p) * inv;
  if (u < 0.0 || u > 1.0) return false;
  const V3 q = cross(s, m.e1[i]);
  v = dot(d, q) * inv;
  if (v < 0.0 || u + v > 1.0) return false;
  t = dot(m.e2[i], q) * inv;
  return true;
}

// Candidate acceptance: in front of the origin by more than t_min (in ray
// parameter units), not the triangle just left, nearest first and the lower
// triangle index on an exact tie.
void consider(const Mesh& m, uint32_t i, V3 o, V3 d, int64_t exclude, double t_min, Hit& best) {
  if ((int64_t)i == exclude) return;
  double t, u, v;
  if (!moller_trumbore(m, i, o, d, t, u, v)) return;
  if (!(t > t_min)) return;
  if (!best.found || t < best.t || (t == best.t && i < best.tri)) {
    best.found = true; best.tri = i; best.t = t; best.u = u; best.v = v;
  }
}

Hit closest_hit_brute(const Mesh& m, V3 o, V3 d, int64_t exclude, double t_min) {
  Hit best;
  for (uint32_t i = 0; i < m.nt; ++i) consider(m, i, o, d, exclude, t_min, best);
  return best;
}

void build_bvh(Mesh& m) {
  m.nodes.clear();
  m.order.resize(m.nt);
  for (uint32_t i = 0; i < m.nt; ++i) m.order[i] = i;
  if (m.nt == 0) return;
  std::vector<V3> centroid(m.nt);
  for (uint32_t i = 0; i < m.nt; ++i) centroid[i] = m.v0[i] + (1.0 / 3.0) * (m.e1[i] + m.e2[i]);
  struct Task { int32_t node; uint32_t first, count; };
  std::vector<Task> stack;
  m.nodes.push_back({});
  stack.push_back({0, 0, m.nt});
  while (!stack.empty()) {
    const Task tk = stack.back();
    stack.pop_back();
    Mesh::Node nd{};
    for (int a = 0; a < 3; ++a) { nd.lo[a] = INFINITY; nd.hi[a] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t k = tk.first; k < tk.first + tk.count; ++k) {
      const uint32_t i = m.order[k];
      const V3 pts[3] = {m.v0[i], m.v0[i] + m.e1[i], m.v0[i] + m.e2[i]};
      for (const V3& p : pts) {
        const double c[3] = {p.x, p.y, p.z};
        for (int a = 0; a < 3; ++a) { nd.lo[a] = std::min(nd.lo[a], c[a]); nd.hi[a] = std::max(nd.hi[a], c[a]); }
      }
      const double c[3] = {centroid[i].x, centroid[i].y, centroid[i].z};
      for (int a = 0; a < 3; ++a) { clo[a] = std::min(clo[a], c[a]); chi[a] = std::max(chi[a], c[a]); }
    }
    // Pad boxes by a relative 1e-9 so that rounding never drops a hit.
    for (int a = 0; a < 3; ++a) {
      const double pad = 1e-9 * (std::fabs(nd.lo[a]) + std::fabs(nd.hi[a]) + 1e-3);
      nd.lo[a] -= pad; nd.hi[a] += pad;
    }
    nd.left = nd.right = -1;
    nd.first = tk.first;
    nd.count = tk.count;
    int axis = 0;
    for (int a = 1; a < 3; ++a) if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    if (tk.count > 4 && chi[axis] > clo[axis]) {
      auto key = [&](uint32_t i) { return axis == 0 ? centroid[i].x : axis == 1 ? centroid[i].y : centroid[i].z; };
      const uint32_t mid = tk.first + tk.count / 2;
      std::nth_element(m.order.begin() + tk.first, m.order.begin() + mid, m.order.begin() + tk.first + tk.count,
                       [&](uint32_t a, uint32_t b) { return key(a) < key(b) || (key(a) == key(b) && a < b); });
      nd.left = (int32_t)m.nodes.size();
      m.nodes.push_back({});
      nd.right = (int32_t)m.nodes.size();
      m.nodes.push_back({});
      stack.push_back({nd.left, tk.first, mid - tk.first});
      stack.push_back({nd.right, mid, tk.first + tk.count - mid});
      nd.count = 0;
    }
    m.nodes[tk.node] = nd;
  }
}

// Slab test: does the ray o + t d, t in [0, t_max], meet the box?
bool ray_box(const Mesh::Node& nd, V3 o, V3 d, double t_max) {
  const double oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
  double t0 = 0.0, t1 = t_max;
  for (int a = 0; a < 3; ++a) {
    if (dd[a] == 0.0) {
      if (oo[a] < nd.lo[a] || oo[a] > nd.hi[a]) return false;
      continue;
    }
    double ta = (nd.lo[a] - oo[a]) / dd[a], tb = (nd.hi[a] - oo[a]) / dd[a];
    if (ta > tb) std::swap(ta, tb);
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
    if (t0 > t1) return false;
  }
  return true;
}

Hit closest_hit_bvh(const Mesh& m, V3 o, V3 d, int64_t exclude, double t_min) {
  Hit best;
  if (m.nodes.empty()) return best;
  std::vector<int32_t> stack;
  stack.reserve(128);
  stack.push_back(0);
  while (!stack.empty()) {
    const Mesh::Node& nd = m.nodes[stack.back()];
    stack.pop_back();
    if (!ray_box(nd, o, d, best.found ? best.t : INFINITY)) continue;
    if (nd.left < 0) {
      for (uint32_t k = nd.first; k < nd.first + nd.count; ++k) consider(m, m.order[k], o, d, exclude, t_min, best);
    } else {
      stack.push_back(nd.left);
      stack.push_back(nd.right);
    }
  }
  return best;
}

Hit closest_hit(const Mesh& m, V3 o, V3 d, int64_t exclude, double t_min, int mode) {
  const bool brute = mode == 1 || (mode == 0 && m.nt <= 5000);
  return brute ? closest_hit_brute(m, o, d, exclude, t_min) : closest_hit_bvh(m, o, d, exclude, t_min);
}

// ---------------------------------------------------------------------------
// Eq. 15: Rodrigues rotation from the free-stream frame (flow along +z) to the
// body frame, about u = z x Vhat by beta = acos(z . Vhat).  Reading of the
// degenerate axes: beta ~ 0 -> identity; beta ~ pi -> half turn about x.
// ---------------------------------------------------------------------------
V3 rodrigues(V3 Vhat, V3 x) {
  const V3 z{0.0, 0.0, 1.0};
  const V3 axis = cross(z, Vhat);
  const double s = norm(axis);
  const double c = std::max(-1.0, std::min(1.0, dot(z, Vhat)));
  if (s < 1e-12) {
    if (c > 0.0) return x;
    return {x.x, -x.y, -x.z};
  }
  const V3 u = (1.0 / s) * axis;
  const double beta = std::acos(c);
  const double cb = std::cos(beta), sb = std::sin(beta);
  return cb * x + sb * cross(u, x) + ((1.0 - cb) * dot(u, x)) * u;
}

// ---------------------------------------------------------------------------
// Gas-surface interaction (§II.A, with the Maxwell diffuse/specular mix named
// in §I).  The diffuse law is read as the flux-weighted half-range Maxwellian
// at the wall temperature: normal speed c_W sqrt(-ln u1), tangential speed
// c_W sqrt(-ln u2) at the angle 2 pi u3 in the triangle frame (t1, n x t1).
// Velocities are in units of the free-stream c_mp; cw = c_W / c_mp.
// ---------------------------------------------------------------------------
V3 gsi(V3 v, V3 nrm, V3 t1, const double u[4], double eps, double cw) {
  if (u[0] < eps) {
    const V3 n_out = dot(v, nrm) < 0.0 ? nrm : (-1.0) * nrm;
    const V3 t2 = cross(nrm, t1);
    const double vn = cw * std::sqrt(-std::log(u[1]));
    const double vt = cw * std::sqrt(-std::log(u[2]));
    const double ang = 2.0 * kPi * u[3];
    return vn * n_out + (vt * std::cos(ang)) * t1 + (vt * std::sin(ang)) * t2;
  }
  return v - (2.0 * dot(v, nrm)) * nrm;
}

// Cercignani-Lampis-Lord surface model (Lord's sampling of the CL kernel; an
// alternative to the Maxwell mix, not used in the paper).  In units of the
// wall's thermal speed c_W, with the hit-side normal n (pointing back into
// the gas), the incident normal speed v_n > 0 and tangential velocity v_t:
//   normal:     r = sqrt(-alpha_n ln u0), theta = 2 pi u1,
//               v_n' = sqrt(r^2 + (1 - alpha_n) v_n^2 + 2 r sqrt(1 - alpha_n) v_n cos theta)
//   tangential: rho = sqrt(-alpha_t ln u2), phi = 2 pi u3,
//               v_t' = sqrt(1 - alpha_t) v_t + rho (cos phi t1 + sin phi t2),
// alpha_n the normal-energy accommodation, alpha_t = sigma_t (2 - sigma_t)
// with sigma_t the tangential-momentum accommodation.  alpha_n = alpha_t = 1
// is the diffuse law above; 0 is specular reflection.
V3 cll(V3 v, V3 nrm, V3 t1, const double u[4], double alpha_n, double alpha_t, double cw) {
  const V3 n_out = dot(v, nrm) < 0.0 ? nrm : (-1.0) * nrm;
  const V3 t2 = cross(nrm, t1);
  const double vn = -dot(v, n_out) / cw;
  const V3 vt = (1.0 / cw) * (v + (cw * vn) * n_out);
  const double r = std::sqrt(-alpha_n * std::log(u[0]));
  const double theta = 2.0 * kPi * u[1];
  const double b = std::sqrt(1.0 - alpha_n) * vn;
  const double vn_out = std::sqrt(std::max(0.0, r * r + b * b + 2.0 * r * b * std::cos(theta)));
  const double rho = std::sqrt(-alpha_t * std::log(u[2]));
  const double phi = 2.0 * kPi * u[3];
  const V3 vt_out = std::sqrt(1.0 - alpha_t) * vt + (rho * std::cos(phi)) * t1 + (rho * std::sin(phi)) * t2;
  return cw * (vn_out * n_out + vt_out);
}

}  // namespace

// ===========================================================================
// C interface (ctypes).  Plain pointers; the caller owns every buffer.
// ===========================================================================
extern "C" {

typedef struct {
  double n, T_inf, m, V;
  double dir[3];
  double T_W, eps_diffuse;
  double A_ref, ref_point[3];
  double r_cv, center[3];
  uint32_t max_bounces;
  uint32_t stream;
  uint64_t seed;
  double t_min_len;     // smallest accepted hit distance in metres (e.g. 1e-9)
  int32_t intersect;    // 0 auto, 1 brute force, 2 median-split BVH
  int32_t threads;      // 0 = all hardware threads
  int32_t cv_kind;      // 0 sphere (Eq. 11, 14a-c); 1 box, flux-weighted faces; 2 box, free-stream Maxwellian faces
  int32_t pad;
  double box_lo[3], box_hi[3];  // box control volume (cv_kind 1, 2), body frame, metres
  double l_ref;                 // moment reference length (<= 0: 1 m)
  int32_t gsi_model;            // 0 Maxwell mix (eps_diffuse), 1 Cercignani-Lampis-Lord (alpha_n, sigma_t)
  int32_t pad2;
  double alpha_n, sigma_t;
} orc_params;

typedef struct {
  double force[3], torque[3];
  double CD, CD_sigma, gamma, weight, S, S_W, q_inf, c_mp;
  double sum_dv[3], sum_rdv[3], sum_d, sum_d2;
  uint64_t n_particles, n_hits, n_hit_particles, n_truncated;
  double CF[3], CM[3];  // force / (q_inf A_ref); torque / (q_inf A_ref l_ref) (§III.D.1)
} orc_result;

// Per-particle records (each pointer may be null; K = hits kept per particle).
typedef struct {
  double* pos;      // [count][3] seeded position, metres
  double* vel;      // [count][3] seeded velocity, c_mp units
  double* dv;       // [count][3] sum of (v_in - v_out) over the particle's hits
  uint32_t* n_hits; // [count]
  uint32_t* truncated; // [count]
  uint32_t* tri;    // [count][K] triangle hit at bounce b (b < K)
  double* bary;     // [count][K] smallest barycentric coordinate of that hit
  double* cosi;     // [count][K] |cos| of the incidence angle of that hit
  double* edge;     // [count][K] distance (m) from that hit point to the triangle's nearest edge
  uint32_t K;
} orc_records;

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }
double orc_uniform(uint32_t w) { return uniform_from_word(w); }
void orc_seed_uniforms(uint64_t seed, uint32_t stream, uint64_t pid, double* out) { seed_uniforms(seed, stream, pid, out); }
double orc_gamma_coefficient(double S) { return gamma_coefficient(S); }
double orc_position_norm(double S) { return position_norm(S); }
double orc_g_phi(double phi, double S) { return g_phi(phi, S); }
double orc_h_x(double x, double S) { return h_x(x, S); }
double orc_position_cdf(double x, double S) { return position_cdf(x, S); }
double orc_position_inverse(double u, double S) { return position_inverse(u, S); }
double orc_normal_speed_norm(double s) { return normal_speed_norm(s); }
double orc_normal_speed_pdf(double x, double s) { return normal_speed_pdf(x, s); }
double orc_normal_speed_cdf(double x, double s) { return normal_speed_cdf(x, s); }
double orc_normal_speed_inverse(double u, double s) { return normal_speed_inverse(u, s); }
double orc_truncated_normal_cdf(double x, double s) { return truncated_normal_cdf(x, s); }
double orc_truncated_normal_inverse(double u, double s) { return truncated_normal_inverse(u, s); }
double orc_flux_G(double s) { return flux_G(s); }
double orc_flux_P(double s) { return flux_P(s); }

void orc_surface_force(const double* nrm, const double* Vhat, double S, double eps, double cw, double* out) {
  store3(out, surface_force(unit(load3(nrm)), unit(load3(Vhat)), S, eps, cw));
}

void orc_cll(const double* v, const double* nrm, const double* t1, const double* u, double alpha_n, double alpha_t,
             double cw, double* out) {
  store3(out, cll(load3(v), unit(load3(nrm)), unit(load3(t1)), u, alpha_n, alpha_t, cw));
}

void orc_rodrigues(const double* Vhat, const double* x, double* out) {
  store3(out, rodrigues(unit(load3(Vhat)), load3(x)));
}

void orc_gsi(const double* v, const double* nrm, const double* t1, const double* u, double eps, double cw,
             double* out) {
  store3(out, gsi(load3(v), load3(nrm), load3(t1), u, eps, cw));
}

// Eq. 4 (Bird): C_D of a convex sphere, diffuse re-emission; S_W = V / c_W.
double orc_sphere_cd_paper(double S, double S_W) {
  return std::exp(-S * S) / (kSqrtPi * S * S * S) * (1.0 + 2.0 * S * S) +
         (4.0 * S * S * S * S + 4.0 * S * S - 1.0) / (2.0 * S * S * S * S) * std::erf(S) +
         2.0 * kSqrtPi / (3.0 * S_W);
}

// Eq. 3 exactly as printed (Sentman's double-sided plate, A_ref = one face).
double orc_plate_cd_paper(double S, double S_W, double alpha) {
  const double sc = S * std::cos(alpha);
  return 2.0 / (kSqrtPi * S) *
         (std::exp(-sc * sc) + kSqrtPi * sc * (1.0 + 1.0 / (2.0 * S * S)) * std::erf(sc) +
          kPi * S / S_W * std::cos(alpha) * std::cos(alpha));
}

// Eq. 3 with the re-emission term re-derived for a double-sided plate: the two
// faces re-emit G(s) - G(-s) = s more molecules on the windward side, so the
// re-emission term is sqrt(pi) cos^2(alpha) / S_W (half the printed term; the
// first three terms are unchanged).
double orc_plate_cd_derived(double S, double S_W, double alpha) {
  const double sc = S * std::cos(alpha);
  return 2.0 / (kSqrtPi * S) * (std::exp(-sc * sc) + kSqrtPi * sc * (1.0 + 1.0 / (2.0 * S * S)) * std::erf(sc)) +
         kSqrtPi * std::cos(alpha) * std::cos(alpha) / S_W;
}

// Gauss-Legendre nodes on [-1,1] by Newton on P_n (Golub-Welsch is not needed).
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1; p1 = p2;
    }
    const double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// C_D of a smooth sphere of radius R (A_ref = pi R^2) by Gauss-Legendre
// quadrature of surface_force over mu = n . Vhat (axisymmetric).
double orc_sphere_cd_quadrature(double S, double eps, double cw, int nodes) {
  std::vector<double> x, w;
  gauss_legendre(nodes, x, w);
  const V3 Vhat{0, 0, 1};
  double drag = 0.0;
  for (int i = 0; i < nodes; ++i) {
    const double mu = x[i];
    const V3 nrm{std::sqrt(std::max(0.0, 1.0 - mu * mu)), 0.0, mu};
    drag += w[i] * 2.0 * kPi * dot(surface_force(nrm, Vhat, S, eps, cw), Vhat);
  }
  return drag / (0.5 * S * S * kPi);
}

// C_D of a smooth closed cylinder (radius R, length L, axis z) at angle alpha
// between the flow and the axis; A_ref = 2 R L.  Side by the trapezoid rule in
// the azimuth (periodic, analytic integrand), end caps as flat discs.
double orc_cylinder_cd_quadrature(double S, double eps, double cw, double alpha, double R, double L, int nodes) {
  const V3 Vhat{std::sin(alpha), 0.0, std::cos(alpha)};
  double drag = 0.0;
  for (int i = 0; i < nodes; ++i) {
    const double psi = 2.0 * kPi * i / nodes;
    const V3 nrm{std::cos(psi), std::sin(psi), 0.0};
    drag += dot(surface_force(nrm, Vhat, S, eps, cw), Vhat) * R * L * (2.0 * kPi / nodes);
  }
  const double cap = kPi * R * R;
  drag += dot(surface_force({0, 0, 1}, Vhat, S, eps, cw), Vhat) * cap;
  drag += dot(surface_force({0, 0, -1}, Vhat, S, eps, cw), Vhat) * cap;
  return drag / (0.5 * S * S * 2.0 * R * L);
}

// Panel sum over a triangulation without shadowing (exact expectation for a
// closed convex mesh with outward winding, or for a single planar sheet when
// two_sided = 1): returns the force in units of n m c^2 (per unit of length^2).
void orc_panel_sum(const double* xyz, const uint32_t* tri, uint32_t nt, int two_sided, const double* Vhat_in,
                   double S, double eps, double cw, double* force_out) {
  const V3 Vhat = unit(load3(Vhat_in));
  V3 F{0, 0, 0};
  for (uint32_t i = 0; i < nt; ++i) {
    const V3 a = load3(xyz + 3 * tri[3 * i]), b = load3(xyz + 3 * tri[3 * i + 1]), c = load3(xyz + 3 * tri[3 * i + 2]);
    const V3 cr = cross(b - a, c - a);
    const double A = 0.5 * norm(cr);
    if (A == 0.0) continue;
    const V3 nrm = unit(cr);
    F = F + A * surface_force(nrm, Vhat, S, eps, cw);
    if (two_sided) F = F + A * surface_force((-1.0) * nrm, Vhat, S, eps, cw);
  }
  store3(force_out, F);
}

// ------------------------------- mesh handle -------------------------------
void* orc_mesh_create(const double* xyz, uint32_t nv, const uint32_t* tri, uint32_t nt) {
  Mesh* m = new Mesh();
  m->nt = nt;
  m->v0.resize(nt); m->e1.resize(nt); m->e2.resize(nt); m->nrm.resize(nt); m->t1.resize(nt); m->area.resize(nt);
  for (uint32_t i = 0; i < nt; ++i) {
    for (int k = 0; k < 3; ++k) if (tri[3 * i + k] >= nv) { delete m; return nullptr; }
    const V3 a = load3(xyz + 3 * tri[3 * i]), b = load3(xyz + 3 * tri[3 * i + 1]), c = load3(xyz + 3 * tri[3 * i + 2]);
    m->v0[i] = a;
    m->e1[i] = b - a;
    m->e2[i] = c - a;
    const V3 cr = cross(m->e1[i], m->e2[i]);
    m->area[i] = 0.5 * norm(cr);
    m->nrm[i] = m->area[i] > 0 ? unit(cr) : V3{0, 0, 0};
    m->t1[i] = norm(m->e1[i]) > 0 ? unit(m->e1[i]) : V3{0, 0, 0};
  }
  build_bvh(*m);
  return m;
}

void orc_mesh_destroy(void* h) { delete (Mesh*)h; }

// Closest hit of one ray (for the intersection pins).  Returns the triangle
// index or -1, and t, u, v.
int64_t orc_closest_hit(const void* h, const double* o, const double* d, int64_t exclude, double t_min, int mode,
                        double* tuv) {
  const Hit hit = closest_hit(*(const Mesh*)h, load3(o), load3(d), exclude, t_min, mode);
  if (tuv) { tuv[0] = hit.t; tuv[1] = hit.u; tuv[2] = hit.v; }
  return hit.found ? (int64_t)hit.tri : -1;
}

// ------------------------------- the TPMC run -------------------------------
// Traces particles [pid_begin, pid_begin + count) of a run of N_total
// particles.  Returns 0 on success, -1 on invalid input.
int orc_trace(const void* mesh_handle, const orc_params* p, uint64_t N_total, uint64_t pid_begin, uint64_t count,
              orc_result* res, double* panel_dv, const orc_records* rec) {
  const Mesh& m = *(const Mesh*)mesh_handle;
  if (!(p->n > 0 && p->T_inf > 0 && p->m > 0 && p->V > 0 && p->T_W > 0)) return -1;
  if (p->cv_kind == 0 && !(p->r_cv > 0)) return -1;
  if (!(p->eps_diffuse >= 0 && p->eps_diffuse <= 1) || p->max_bounces < 1 || N_total == 0) return -1;
  if (count == 0 || pid_begin + count > N_total) return -1;
  const V3 Vraw = load3(p->dir);
  if (!(norm(Vraw) > 0)) return -1;
  const V3 Vhat = unit(Vraw);

  // a1: free-stream set-up (Nomenclature; Eq. 10; §II.A particle weight).
  const double c = std::sqrt(2.0 * kBoltzmann * p->T_inf / p->m);
  const double cW = std::sqrt(2.0 * kBoltzmann * p->T_W / p->m);
  const double S = p->V / c;
  const double cw = cW / c;
  if (p->cv_kind < 0 || p->cv_kind > 2) return -1;
  if (p->gsi_model < 0 || p->gsi_model > 1) return -1;
  if (p->gsi_model == 1 && !(p->alpha_n >= 0 && p->alpha_n <= 1 && p->sigma_t >= 0 && p->sigma_t <= 1)) return -1;
  const double alpha_t = p->sigma_t * (2.0 - p->sigma_t);
  const bool box = p->cv_kind != 0;
  // Rectangular control volume (§I, §III.A): faces f = 2 a + k are x_a = hi_a
  // (k = 0, inward normal -e_a) and x_a = lo_a (k = 1, inward normal +e_a).
  // Face f receives the flat-plate number flux A_f n c G(s_f) of the free
  // stream, s_f = S (Vhat . inward normal), and the particle ids
  // [floor(N C_f), floor(N C_{f+1})), C_f the cumulative share of the total.
  struct Face { int axis; double coord; V3 n_in; double s, area; uint64_t begin, end; };
  Face faces[6];
  double box_flux = 0.0;  // sum of A_f G(s_f), m^2
  if (box) {
    for (int a = 0; a < 3; ++a)
      if (!(p->box_hi[a] > p->box_lo[a])) return -1;
    for (int f = 0; f < 6; ++f) {
      Face& F = faces[f];
      F.axis = f / 2;
      const int a1 = (F.axis + 1) % 3, a2 = (F.axis + 2) % 3;
      const double sign = (f % 2 == 0) ? -1.0 : 1.0;
      F.coord = (f % 2 == 0) ? p->box_hi[F.axis] : p->box_lo[F.axis];
      F.n_in = V3{F.axis == 0 ? sign : 0.0, F.axis == 1 ? sign : 0.0, F.axis == 2 ? sign : 0.0};
      F.s = S * dot(Vhat, F.n_in);
      F.area = (p->box_hi[a1] - p->box_lo[a1]) * (p->box_hi[a2] - p->box_lo[a2]);
      box_flux += F.area * flux_G(F.s);
    }
    double cum = 0.0;
    for (int f = 0; f < 6; ++f) {
      faces[f].begin = (uint64_t)std::floor((double)N_total * cum);
      cum += faces[f].area * flux_G(faces[f].s) / box_flux;
      faces[f].end = f == 5 ? N_total : (uint64_t)std::floor((double)N_total * cum);
    }
  }
  const double gamma = box ? box_flux * c * p->n
                           : gamma_coefficient(S) * c * p->n * p->r_cv * p->r_cv;  // molecules per second
  const double weight = gamma / (double)N_total;                                   // molecules/s per particle
  const double q_inf = 0.5 * p->n * p->m * p->V * p->V;
  const V3 center = load3(p->center), ref = load3(p->ref_point);

  int threads = p->threads > 0 ? p->threads : (int)std::max(1u, std::thread::hardware_concurrency());
  if ((uint64_t)threads > std::max<uint64_t>(count, 1)) threads = (int)std::max<uint64_t>(count, 1);

  struct Acc {
    double dv[3] = {0, 0, 0}, rdv[3] = {0, 0, 0}, d = 0, d2 = 0;
    double dv_c[3] = {0, 0, 0}, rdv_c[3] = {0, 0, 0}, d_c = 0, d2_c = 0;  // Neumaier compensations
    uint64_t hits = 0, hit_particles = 0, truncated = 0;
    std::vector<double> panel;
  };
  auto neumaier = [](double& sum, double& comp, double x) {
    const double t = sum + x;
    if (std::fabs(sum) >= std::fabs(x)) comp += (sum - t) + x; else comp += (x - t) + sum;
    sum = t;
  };
  std::vector<Acc> acc(threads);
  const double t_min_len = p->t_min_len;

  auto work = [&](int tid) {
    Acc& A = acc[tid];
    if (panel_dv) A.panel.assign((size_t)m.nt * 3, 0.0);
    const uint64_t lo = count * (uint64_t)tid / threads, hi = count * (uint64_t)(tid + 1) / threads;
    for (uint64_t k = lo; k < hi; ++k) {
      const uint64_t pid = pid_begin + k;
      double us[5];
      seed_uniforms(p->seed, p->stream, pid, us);
      const double* u0 = us;       // u_x, u_theta, u_vn, u_r
      const double* u1 = us + 4;   // u_a
      V3 pos, v;
      if (box) {
        // Rectangular CV: the face owning this id; a uniform point on it;
        // the inward normal speed from the face's law; tangential components
        // of the free stream plus thermal parts (Box-Muller, as on the sphere).
        int f = 0;
        while (f < 5 && pid >= faces[f].end) ++f;
        const Face& F = faces[f];
        const int a1 = (F.axis + 1) % 3, a2 = (F.axis + 2) % 3;
        double pc[3];
        pc[F.axis] = F.coord;
        pc[a1] = p->box_lo[a1] + u0[0] * (p->box_hi[a1] - p->box_lo[a1]);
        pc[a2] = p->box_lo[a2] + u0[1] * (p->box_hi[a2] - p->box_lo[a2]);
        pos = V3{pc[0], pc[1], pc[2]};
        const double vn = p->cv_kind == 1 ? normal_speed_inverse(u0[2], F.s) : truncated_normal_inverse(u0[2], F.s);
        const double rad = std::sqrt(-std::log(u0[3]));
        const double vh[3] = {Vhat.x, Vhat.y, Vhat.z};
        double vc[3];
        vc[F.axis] = 0.0;
        vc[a1] = S * vh[a1] + rad * std::cos(2.0 * kPi * u1[0]);
        vc[a2] = S * vh[a2] + rad * std::sin(2.0 * kPi * u1[0]);
        v = vn * F.n_in + V3{vc[0], vc[1], vc[2]};
      } else {
      // a3: position on the control sphere (Eq. 11 by inverse transform,
      // theta uniform); stream frame has the flow along +z, so the upstream
      // pole phi = pi/2 sits at -z.
      const double x = position_inverse(u0[0], S);
      const double cphi = std::sqrt((1.0 - x) * (1.0 + x));
      const double theta = 2.0 * kPi * u0[1];
      const V3 out_s{cphi * std::cos(theta), cphi * std::sin(theta), -x};
      const V3 out_b = rodrigues(Vhat, out_s);  // a5 (Eq. 15)
      pos = center + p->r_cv * out_b;
      // a4: local frame n (inward), t1 (tangential projection of the flow),
      // t2 = t1 x n; velocity components from Eq. 14a-c; then the transpose
      // of the local frame matrix carries them to body coordinates.
      const V3 nl = (-1.0) * out_b;
      V3 t1 = Vhat - dot(Vhat, nl) * nl;
      t1 = norm(t1) > 1e-300 ? unit(t1) : rodrigues(Vhat, V3{std::cos(theta), std::sin(theta), 0.0});
      const V3 t2 = cross(t1, nl);
      const double s_n = S * x;
      const double vn = normal_speed_inverse(u0[2], s_n);
      const double rad = std::sqrt(-std::log(u0[3]));
      const double vt1 = S * cphi + rad * std::cos(2.0 * kPi * u1[0]);
      const double vt2 = rad * std::sin(2.0 * kPi * u1[0]);
      v = vn * nl + vt1 * t1 + vt2 * t2;
      }
      if (rec) {
        if (rec->pos) store3(rec->pos + 3 * k, pos);
        if (rec->vel) store3(rec->vel + 3 * k, v);
      }
      // a6-a9: closest hit, re-emission, momentum sum, until a miss.
      V3 dv_p{0, 0, 0}, rdv_p{0, 0, 0};
      uint32_t nh = 0;
      bool trunc = true;
      int64_t last = -1;
      for (uint32_t b = 0; b < p->max_bounces; ++b) {
        const double t_min = t_min_len / norm(v);
        const Hit hit = closest_hit(m, pos, v, last, t_min, p->intersect);
        if (!hit.found) { trunc = false; break; }
        const uint32_t i = hit.tri;
        const V3 hp = pos + hit.t * v;
        double ub[4];
        draw_block(p->seed, p->stream, pid, 2 + b, ub);
        const V3 v_out = p->gsi_model == 1 ? cll(v, m.nrm[i], m.t1[i], ub, p->alpha_n, alpha_t, cw)
                                           : gsi(v, m.nrm[i], m.t1[i], ub, p->eps_diffuse, cw);
        const V3 dvh = v - v_out;
        dv_p = dv_p + dvh;
        rdv_p = rdv_p + cross(hp - ref, dvh);
        if (panel_dv) for (int a = 0; a < 3; ++a) A.panel[3 * i + a] += (a == 0 ? dvh.x : a == 1 ? dvh.y : dvh.z);
        if (rec && b < rec->K) {
          if (rec->tri) rec->tri[(size_t)k * rec->K + b] = i;
          if (rec->bary) rec->bary[(size_t)k * rec->K + b] = std::min({hit.u, hit.v, 1.0 - hit.u - hit.v});
          if (rec->cosi) rec->cosi[(size_t)k * rec->K + b] = std::fabs(dot(unit(v), m.nrm[i]));
          if (rec->edge) {
            // distance to the edge opposite vertex j = (barycentric of j) x (height over that edge)
            const double twoA = 2.0 * m.area[i];
            const double w0 = 1.0 - hit.u - hit.v;
            const double d0 = w0 * twoA / norm(m.e2[i] - m.e1[i]);
            const double d1 = hit.u * twoA / norm(m.e2[i]);
            const double d2 = hit.v * twoA / norm(m.e1[i]);
            rec->edge[(size_t)k * rec->K + b] = std::min({d0, d1, d2});
          }
        }
        ++nh;
        pos = hp;
        v = v_out;
        last = i;
      }
      if (rec) {
        if (rec->dv) store3(rec->dv + 3 * k, dv_p);
        if (rec->n_hits) rec->n_hits[k] = nh;
        if (rec->truncated) rec->truncated[k] = trunc ? 1u : 0u;
      }
      const double d = dot(dv_p, Vhat);
      const double dva[3] = {dv_p.x, dv_p.y, dv_p.z}, rdva[3] = {rdv_p.x, rdv_p.y, rdv_p.z};
      for (int a = 0; a < 3; ++a) { neumaier(A.dv[a], A.dv_c[a], dva[a]); neumaier(A.rdv[a], A.rdv_c[a], rdva[a]); }
      neumaier(A.d, A.d_c, d);
      neumaier(A.d2, A.d2_c, d * d);
      A.hits += nh;
      A.hit_particles += nh > 0;
      A.truncated += trunc;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto& th : pool) th.join();

  // a10: fixed-order combination and the final FP64 reduction.
  double sdv[3] = {0, 0, 0}, srdv[3] = {0, 0, 0}, sd = 0, sd2 = 0;
  double cdv[3] = {0, 0, 0}, crdv[3] = {0, 0, 0}, cd = 0, cd2 = 0;
  uint64_t hits = 0, hitp = 0, trunc = 0;
  for (const Acc& A : acc) {
    for (int a = 0; a < 3; ++a) {
      neumaier(sdv[a], cdv[a], A.dv[a] + A.dv_c[a]);
      neumaier(srdv[a], crdv[a], A.rdv[a] + A.rdv_c[a]);
    }
    neumaier(sd, cd, A.d + A.d_c);
    neumaier(sd2, cd2, A.d2 + A.d2_c);
    hits += A.hits; hitp += A.hit_particles; trunc += A.truncated;
  }
  for (int a = 0; a < 3; ++a) { sdv[a] += cdv[a]; srdv[a] += crdv[a]; }
  sd += cd; sd2 += cd2;
  if (panel_dv) {
    for (size_t j = 0; j < (size_t)m.nt * 3; ++j) {
      double s = 0, cc = 0;
      for (const Acc& A : acc) neumaier(s, cc, A.panel[j]);
      panel_dv[j] = s + cc;
    }
  }

  // Force = (molecules/s per particle) x m x c x sum(dv) (§II.A); C_D from
  // Eq. 1.  A run over a subset of the particle ids estimates the same force
  // from the particles it traced, so the weight is Gamma / count there.
  const double scale = gamma / (double)count * p->m * c;
  for (int a = 0; a < 3; ++a) { res->force[a] = scale * sdv[a]; res->torque[a] = scale * srdv[a]; }
  res->CD = (res->force[0] * Vhat.x + res->force[1] * Vhat.y + res->force[2] * Vhat.z) / (q_inf * p->A_ref);
  const double l_ref = p->l_ref > 0.0 ? p->l_ref : 1.0;
  for (int a = 0; a < 3; ++a) {
    res->CF[a] = res->force[a] / (q_inf * p->A_ref);
    res->CM[a] = res->torque[a] / (q_inf * p->A_ref * l_ref);
  }
  // Standard error of the mean of the per-particle drag contributions.
  const double nc = (double)count;
  const double mean = sd / nc;
  const double var = count > 1 ? std::max(0.0, (sd2 - nc * mean * mean) / (nc - 1.0)) : 0.0;
  const double k_cd = gamma * p->m * c / (q_inf * p->A_ref);  // C_D per unit mean drag dv
  res->CD_sigma = k_cd * std::sqrt(var / nc);
  res->gamma = gamma;
  res->weight = weight;
  res->S = S;
  res->S_W = p->V / cW;
  res->q_inf = q_inf;
  res->c_mp = c;
  for (int a = 0; a < 3; ++a) { res->sum_dv[a] = sdv[a]; res->sum_rdv[a] = srdv[a]; }
  res->sum_d = sd;
  res->sum_d2 = sd2;
  res->n_particles = count;
  res->n_hits = hits;
  res->n_hit_particles = hitp;
  res->n_truncated = trunc;
  return 0;
}

}  // extern "C"
