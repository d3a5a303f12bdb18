// CUDA kernels of the TPMC hot path for sm_103a (GB300).
//
//   setup_kernel     FP64: free-stream set-up per query (Nomenclature; Eq. 10
//                    flux; particle weight, §II.A), Rodrigues matrix (Eq. 15),
//                    fixed-point scale, start table of the latitude inverse CDF.
//   trace_kernel<R, MINB, CLL, W, COUNT>
//                    persistent, one warp = 32 particle slots refilled from a
//                    global work counter by ballot; per slot: Philox draws,
//                    seeding (Eq. 11, Eq. 14a-c, Eq. 15; or the box CV),
//                    BVH closest hit with a watertight ray/triangle test
//                    (§II.A), Maxwell (or, with CLL, Cercignani-Lampis-Lord)
//                    re-emission, int64 fixed-point momentum sums, until the
//                    particle misses or reaches max_bounces.  R = float (FP32
//                    path) or double; MINB = register-capped occupancy; CLL:
//                    with the CLL branch; W: BVH width; COUNT: with the
//                    node-visit and triangle-test counters and the
//                    per-particle records (verification launches).
//   finalize_kernel  FP64 reduction to force, torque, C_D and its error.
//   panels_kernel    FP64 per-triangle pressure and shear.
//
// This file shares nothing with the CPU oracle; both follow the paper and the
// published Philox4x32-10 definition (Salmon et al., SC'11).
#include <algorithm>
#include <type_traits>

#include <cuda_runtime.h>
#include <math_constants.h>

#include "tpmc_internal.h"

namespace tpmc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kBoltz = 1.380649e-23;
constexpr double kSqrtPiD = 1.7724538509055160273;

// ------------------------------------------------------------------ Philox
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// (k + 1/2) 2^-23 for the top 23 bits k: exact in float and double.
template <typename R>
__device__ __forceinline__ R uniform(uint32_t w) {
  return (R)(w >> 9) * (R)1.1920928955078125e-07 + (R)5.9604644775390625e-08;
}

__device__ __forceinline__ uint4 draws(const QueryDev& q, uint64_t pid, uint32_t block) {
  return philox4x32_10(make_uint4((uint32_t)pid, (uint32_t)(pid >> 32), q.stream_id, block),
                       make_uint2((uint32_t)q.seed, (uint32_t)(q.seed >> 32)));
}

// ----------------------------------------------------------- math by type
template <typename R> struct Fn;
template <> struct Fn<float> {
  static __device__ __forceinline__ float exp(float x) { return expf(x); }
  static __device__ __forceinline__ float log(float x) { return logf(x); }
  static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float erfc(float x) { return erfcf(x); }
  static __device__ __forceinline__ float erfcx(float x) { return erfcxf(x); }
  static __device__ __forceinline__ float ncdfinv(float x) { return normcdfinvf(x); }
  static __device__ __forceinline__ float erfcinv(float x) { return erfcinvf(x); }
  static __device__ __forceinline__ void sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
  static __device__ __forceinline__ float fabs(float x) { return fabsf(x); }
  // The hardware reciprocal (within one unit in the last place), not the
  // correctly rounded division: for the ray's slab constants, the shear
  // constant and hit distances, where the correctly rounded form cost 1-6 %
  // of throughput.  Box tests stay conservative (the builder widens every box
  // by a grid step, far more than these errors move a slab), and the
  // watertight test stays watertight (one shear for all triangles of a ray).
  static __device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
  }
  static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
};
template <> struct Fn<double> {
  static __device__ __forceinline__ double exp(double x) { return ::exp(x); }
  static __device__ __forceinline__ double log(double x) { return ::log(x); }
  static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  static __device__ __forceinline__ double erfc(double x) { return ::erfc(x); }
  static __device__ __forceinline__ double erfcx(double x) { return ::erfcx(x); }
  static __device__ __forceinline__ double ncdfinv(double x) { return ::normcdfinv(x); }
  static __device__ __forceinline__ double erfcinv(double x) { return ::erfcinv(x); }
  static __device__ __forceinline__ void sincospi(double x, double* s, double* c) { ::sincospi(x, s, c); }
  static __device__ __forceinline__ double fabs(double x) { return ::fabs(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
  static constexpr double kTolLat = 1e-14;
  static constexpr double kTolSpeed = 1e-14;
  static constexpr int kIter = 40;
};

// Query constants in the path's precision.
template <typename R> struct QC;
template <> struct QC<float> {
  float S, cw, r_cv, sqrtpi_4S, K1, Dinv, scale;
  float Rm[9], vhat[3], center[3], ref[3];
  __device__ __forceinline__ void load(const QueryDev& q) {
    S = q.fc[kFcS]; cw = q.fc[kFcCw]; r_cv = q.fc[kFcRcv]; sqrtpi_4S = q.fc[kFcSqrtpi4S];
    K1 = q.fc[kFcK1]; Dinv = q.fc[kFcDinv]; scale = q.fc[kFcScale];
#pragma unroll
    for (int i = 0; i < 9; ++i) Rm[i] = q.fc[kFcR + i];
#pragma unroll
    for (int i = 0; i < 3; ++i) { vhat[i] = q.fc[kFcVhat + i]; center[i] = q.fc[kFcCenter + i]; ref[i] = q.fc[kFcRef + i]; }
  }
};
template <> struct QC<double> {
  double S, cw, r_cv, sqrtpi_4S, K1, Dinv, scale;
  double Rm[9], vhat[3], center[3], ref[3];
  __device__ __forceinline__ void load(const QueryDev& q) {
    S = q.S; cw = q.cw; r_cv = q.r_cv; sqrtpi_4S = kSqrtPiD / (4.0 * q.S); K1 = q.K1; Dinv = 1.0 / q.Dnorm;
    scale = 1.0 / q.quantum;
#pragma unroll
    for (int i = 0; i < 9; ++i) Rm[i] = q.R[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) { vhat[i] = q.vhat[i]; center[i] = q.center[i]; ref[i] = q.ref[i]; }
  }
};

// ------------------------------------------------------- seeding (§III.A)
// Latitude law (Eq. 11) in x = sin(phi): CDF written with erfc(-S x) = 1 + erf(S x):
//   H(x) = [ sqrt(pi)/(4S) (2 S^2 x^2 + 1) erfc(-S x) + (x/2) e^{-S^2 x^2} - K1 ] / D,
//   K1 = sqrt(pi)/(4S) (2 S^2 + 1) erfc(S) - e^{-S^2}/2,  so H(-1) = 0 exactly in the algebra.
// Its density h(x) = [e^{-S^2 x^2} + sqrt(pi) S x erfc(-S x)] / D.
template <typename R>
__device__ __forceinline__ R latitude_cdf(R x, R S, R sqrtpi_4S, R K1, R Dinv) {
  const R Sx = S * x;
  return (sqrtpi_4S * ((R)2 * Sx * Sx + (R)1) * Fn<R>::erfc(-Sx) + (R)0.5 * x * Fn<R>::exp(-Sx * Sx) - K1) * Dinv;
}
template <typename R>
__device__ __forceinline__ R latitude_pdf(R x, R S, R Dinv) {
  const R Sx = S * x;
  return (Fn<R>::exp(-Sx * Sx) + (R)kSqrtPiD * Sx * Fn<R>::erfc(-Sx)) * Dinv;
}

// Interpolated start from a table laid out in z = Phi^-1(u).
__device__ __forceinline__ float z_table_start(const float* tab, int n, float z, float z_lo, float z_step) {
  const float f = (z - z_lo) / z_step;
  const int j = min(max((int)floorf(f), 0), n - 2);
  const float w = fminf(fmaxf(f - (float)j, 0.0f), 1.0f);
  return (1.0f - w) * __ldg(&tab[j]) + w * __ldg(&tab[j + 1]);
}

// Float latitude solve near a pole, in w = 1 - x (up) or w = 1 + x (down).
// The probability within w of the pole is the integral of h over that end
// interval; with g = D h, g' = sqrt(pi) S erfc(-S t) and g'' = 2 S^2 e^{-S^2 t^2},
// it is the cubic c0 w + c1 w^2 + c2 w^3 (Taylor, next term below 3e-7
// relative for w < 0.002), coefficients per query from the FP64 set-up.
// Newton from w = q / c0, one step: w, and cos(phi) = sqrt(w (2 - w)), to
// ~1e-7 relative, which x itself cannot carry in float this close to +-1.
// Returns (x, cos(phi)) by value: an out-of-line call that wrote through a
// pointer would keep the caller's variable in local memory.
__device__ __noinline__ float2 latitude_pole(float q, float c0, float c1, float c2, bool up) {
  float w = q / c0;
  const float f = ((c2 * w + c1) * w + c0) * w - q;
  const float d = (3.0f * c2 * w + 2.0f * c1) * w + c0;
  w = fminf(fmaxf(w - f / d, 0.0f), 1.0f);
  return make_float2(up ? 1.0f - w : w - 1.0f, sqrtf(w * (2.0f - w)));
}

constexpr float kPoleW = 0.002f;  // pole solves within this distance of x = +-1

// x = H^-1(u), and cphi = cos(phi) = sqrt(1 - x^2).  Float: start from the
// query's table at z = Phi^-1(u) (error ~1e-4), then one Newton step (error
// ~1e-7 over all tails): a fixed step count keeps the warp converged; within
// kPoleW of a pole, the pole solve above.  Double: the same start, then a
// safeguarded Newton loop (on log H in the lower tail) to double precision.
template <typename R>
__device__ R latitude_inverse(R u, const QueryDev& q, const QC<R>& c, R* cphi) {
  const float z = normcdfinvf((float)u);
  R x = (R)z_table_start(q.htab, kHTable + 1, z, (float)kZLo, (float)((kZHi - kZLo) / kHTable));
  if constexpr (sizeof(R) == 4) {
    const R H = latitude_cdf<R>(x, c.S, c.sqrtpi_4S, c.K1, c.Dinv);
    const R h = latitude_pdf<R>(x, c.S, c.Dinv);
    if (h > (R)0) x -= (H - u) / h;
    x = fmin(fmax(x, (R)-1), (R)1);
    *cphi = Fn<R>::sqrt(((R)1 - x) * ((R)1 + x));
    // within kPoleW of a pole, the pole solve (rare; the common path stays branch-free)
    if (x > 1.0f - kPoleW || x < kPoleW - 1.0f) {
      const bool up = x > 0.0f;
      const int k = up ? kFcPole : kFcPole + 3;
      const float2 r = latitude_pole(up ? 1.0f - u : u, q.fc[k], q.fc[k + 1], q.fc[k + 2], up);
      x = r.x;
      *cphi = r.y;
    }
    return x;
  } else {
    R lo = -1, hi = 1;
    const bool logmode = u < (R)0.0625;
    const R lu = logmode ? Fn<R>::log(u) : (R)0;
#pragma unroll 1
    for (int it = 0; it < Fn<R>::kIter; ++it) {
      const R H = latitude_cdf<R>(x, c.S, c.sqrtpi_4S, c.K1, c.Dinv);
      const R h = latitude_pdf<R>(x, c.S, c.Dinv);
      R f, dx;
      if (logmode) {
        if (!(H > (R)0)) { lo = x; x = (R)0.5 * (lo + hi); continue; }
        f = Fn<R>::log(H) - lu;
        dx = -f * H / h;
      } else {
        f = H - u;
        dx = -f / h;
      }
      if (f == (R)0) break;
      if (f < (R)0) lo = x; else hi = x;
      if (Fn<R>::fabs(dx) <= Fn<R>::kTolLat * (Fn<R>::fabs(x) + (R)1e-3)) { x += dx; break; }
      x += dx;
      if (!(x > lo && x < hi)) x = (R)0.5 * (lo + hi);
    }
    x = fmin(fmax(x, (R)-1), (R)1);
    *cphi = Fn<R>::sqrt(((R)1 - x) * ((R)1 + x));
    return x;
  }
}

// Inward normal speed (Eq. 14a, numerator read as 2 v_n/c_mp): x = v_n/c_mp > 0
// with density p(x) = 2 x e^{-(x-s)^2} / Z(s), Z(s) = e^{-s^2} + sqrt(pi) s erfc(-s).
// The root of F(x) = u is found on the smaller tail, so that the solved
// probability keeps its digits in float:
//   u > 1/2: Q(x) = 1 - F(x) = [e^{-y^2} + sqrt(pi) s erfc(y)] / Z, y = x - s
//            (for s < 0 as e^{-x(x-2s)} [1 + sqrt(pi) s erfcx(y)] / [1 + sqrt(pi) s erfcx(-s)]);
//   u <= 1/2: F(x) by 4-point Gauss-Legendre on [0, x] near x = 0 (F ~ x^2 there), else
//            F = [g(s - x) - g(s)] / Z with g(w) = sqrt(pi) s erfc(w) - e^{-w^2}
//            (for s < 0 as 1 - Q).
// Newton runs on log Q (additive steps) or log F (multiplicative steps in x,
// exact for the x^2 law near 0), inside a bisection bracket.
template <typename R>
__device__ R normal_speed_inverse_adaptive(R u, R s, R x_start) {
  const R sp = (R)kSqrtPiD * s;
  const bool upper = u > (R)0.5;
  const R target = upper ? (R)1 - u : u;  // 1 - u is exact for u = (2k+1) 2^-24
  const R lt = Fn<R>::log(target);
  R Z, Zs;  // Z, and Zs = Z e^{s^2} when s < 0
  if (s >= (R)0) { Z = Fn<R>::exp(-s * s) + sp * Fn<R>::erfc(-s); Zs = Z; }
  else { Zs = (R)1 + sp * Fn<R>::erfcx(-s); Z = Zs; }
  const R xq = fmin((R)0.05, (R)0.3 / ((R)1 + Fn<R>::fabs(s)));
  const R g_s = sp * Fn<R>::erfc(s) - Fn<R>::exp(-s * s);
  R lo = 0, hi = fmax(s, (R)0) + (R)6.5;
  R x = x_start;
  if (!(x > lo && x < hi)) x = (R)0.5 * (lo + hi);
#pragma unroll 1
  for (int it = 0; it < Fn<R>::kIter; ++it) {
    const R y = x - s;
    R T, p;
    if (s >= (R)0) {
      const R e = Fn<R>::exp(-y * y);
      p = (R)2 * x * e / Z;
      if (upper) {
        T = (e + sp * Fn<R>::erfc(y)) / Z;
      } else if (x < xq) {
        const R gx[4] = {(R)0.06943184420297371, (R)0.33000947820757187, (R)0.6699905217924281, (R)0.9305681557970262};
        const R gw[4] = {(R)0.17392742256872692, (R)0.3260725774312731, (R)0.3260725774312731, (R)0.17392742256872692};
        R acc = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const R t = x * gx[k];
          acc += gw[k] * (R)2 * t * Fn<R>::exp(-(t - s) * (t - s));
        }
        T = x * acc / Z;
      } else {
        const R w = s - x;
        T = ((sp * Fn<R>::erfc(w) - Fn<R>::exp(-w * w)) - g_s) / Z;
      }
    } else {
      const R e = Fn<R>::exp(-x * (x - (R)2 * s));
      p = (R)2 * x * e / Zs;
      if (upper) {
        T = e * ((R)1 + sp * Fn<R>::erfcx(y)) / Zs;
      } else if (x < xq) {
        const R gx[4] = {(R)0.06943184420297371, (R)0.33000947820757187, (R)0.6699905217924281, (R)0.9305681557970262};
        const R gw[4] = {(R)0.17392742256872692, (R)0.3260725774312731, (R)0.3260725774312731, (R)0.17392742256872692};
        R acc = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const R t = x * gx[k];
          acc += gw[k] * (R)2 * t * Fn<R>::exp(-t * (t - (R)2 * s));
        }
        T = x * acc / Zs;
      } else {
        T = (Zs - e * ((R)1 + sp * Fn<R>::erfcx(y))) / Zs;
      }
    }
    if (!(T > (R)0)) {
      // underflow or cancellation: x lies deep in the solved tail
      if (upper) hi = x; else lo = x;
      x = (R)0.5 * (lo + hi);
      continue;
    }
    const R f = Fn<R>::log(T) - lt;
    if (f == (R)0) break;
    R dx;
    if (upper) {  // Q decreases in x
      if (f > (R)0) lo = x; else hi = x;
      if (!(p > (R)0)) { x = (R)0.5 * (lo + hi); continue; }
      dx = f * T / p;
    } else {      // F increases in x; Newton in log x
      if (f < (R)0) lo = x; else hi = x;
      if (!(p > (R)0)) { x = (R)0.5 * (lo + hi); continue; }
      dx = x * (Fn<R>::exp(-f * T / (x * p)) - (R)1);
    }
    if (Fn<R>::fabs(dx) <= Fn<R>::kTolSpeed * (x + (R)1e-3)) { x += dx; break; }
    x += dx;
    if (!(x > lo && x < hi)) x = (R)0.5 * (lo + hi);
  }
  return fmax(x, (R)0);
}

// Start of the normal-speed solve from the context's table at (s, z = Phi^-1(u));
// beyond the table's s range: the Gaussian limit s + z / sqrt(2) + 1/(2s)
// (large s) or the small-x law F ~ x^2 / (Z e^{s^2}) (very negative s).
__device__ __forceinline__ float normal_speed_start(const float* tab, float s, float z, float u) {
  const float fs = (s - (float)kVnSLo) / (float)kVnStep;
  if (!(fs <= (float)(kVnNS - 1))) return s + 0.70710678f * z + 0.5f / s;  // also catches NaN
  if (!(fs >= 0.0f)) {
    const float a = -s;
    const float zs = 1.0f - 1.77245385f * a * erfcxf(a);  // e^{s^2} Z
    return fmaxf(sqrtf(u * fmaxf(zs, 1e-30f)), 1e-30f);
  }
  const int i = min((int)fs, kVnNS - 2);
  const float a = fminf(fs - (float)i, 1.0f);
  const float fz = (z - (float)kZLo) / (float)kVnStep;
  const int j = min(max((int)floorf(fz), 0), kVnNZ - 2);
  const float b = fminf(fmaxf(fz - (float)j, 0.0f), 1.0f);
  const float* r0 = tab + i * kVnNZ + j;
  const float* r1 = r0 + kVnNZ;
  const float x = (1.0f - a) * ((1.0f - b) * __ldg(r0) + b * __ldg(r0 + 1)) + a * ((1.0f - b) * __ldg(r1) + b * __ldg(r1 + 1));
  return fmaxf(x, 1e-30f);
}

// Float: one Newton step from the bilinear table start (start error ~3e-5;
// after the step ~6e-8 relative in the median, 2e-5 at the 99th percentile,
// <= 1.5e-4 at the extreme uniforms u ~ 2^-24), on the survival function
// above the median and on the CDF below it (selected per lane, no branch on
// the tail); near x = 0 the CDF comes from 4-point Gauss-Legendre.
// Double: the table start, then the adaptive loop to double precision.
template <typename R>
__device__ R normal_speed_inverse(R u, R s, const float* tab) {
  const float z = normcdfinvf((float)u);
  const R x0 = (R)normal_speed_start(tab, (float)s, z, (float)u);
  if constexpr (sizeof(R) == 8) {
    return normal_speed_inverse_adaptive<R>(u, s, x0);
  } else {
    const float sp = 1.77245385090551602730f * s;
    const bool upper = u > 0.5f;
    const float target = upper ? 1.0f - u : u;
    float Z, Zs, gs = 0.0f;
    if (s >= 0.0f) {
      const float es = expf(-s * s), ecs = erfcf(s);  // erfc(-s) = 2 - erfc(s), in [1, 2]
      Z = es + sp * (2.0f - ecs);
      Zs = Z;
      gs = sp * ecs - es;
    } else {
      Zs = 1.0f + sp * erfcxf(-s);
      Z = Zs;
    }
    const float xq = fminf(0.05f, 0.3f / (1.0f + fabsf(s)));
    float x = x0;
    {
      const float y = x - s;
      float T, p;
      if (s >= 0.0f) {
        const float e = expf(-y * y);
        p = 2.0f * x * e / Z;
        const float ec = erfcf(fabsf(y));
        const float erfc_y = y >= 0.0f ? ec : 2.0f - ec;
        const float erfc_w = y >= 0.0f ? 2.0f - ec : ec;
        T = upper ? (e + sp * erfc_y) / Z : ((sp * erfc_w - e) - gs) / Z;
      } else {
        const float e = expf(-x * (x - 2.0f * s));
        p = 2.0f * x * e / Zs;
        const float qn = e * (1.0f + sp * erfcxf(y));
        T = upper ? qn / Zs : (Zs - qn) / Zs;
      }
      if (!upper && x < xq) {
        // F near x = 0 by quadrature of p on [0, x] (F ~ x^2 keeps its digits)
        const float gx[4] = {0.06943184420297371f, 0.33000947820757187f, 0.6699905217924281f, 0.9305681557970262f};
        const float gw[4] = {0.17392742256872692f, 0.3260725774312731f, 0.3260725774312731f, 0.17392742256872692f};
        // integrand scaled by e^{s^2} when s < 0 (then divided by Zs = Z e^{s^2})
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float t = x * gx[k];
          acc += gw[k] * 2.0f * t * expf(s >= 0.0f ? -(t - s) * (t - s) : -t * (t - 2.0f * s));
        }
        T = x * acc / (s >= 0.0f ? Z : Zs);
      }
      const float f = T - target;
      const float dx = p > 0.0f ? (upper ? f / p : -f / p) : 0.0f;
      const float xn = x + dx;
      x = xn > 0.0f ? xn : 0.5f * x;
    }
    return x;
  }
}

// Seed particle pid of query q: position on the CV (body frame, m) and
// velocity (c_mp units).  Stream frame: flow along +z, upstream pole at -z;
// local frame n (inward), t1 (tangential projection of the flow), t2 = t1 x n;
// Eq. 14b-c tangential laws by Box-Muller; Eq. 15 rotation to the body frame.
// Box-CV constants in the path's precision.
template <typename R> struct BoxC;
template <> struct BoxC<float> {
  static __device__ __forceinline__ float s(const QueryDev& q, int f) { return q.fface_s[f]; }
  static __device__ __forceinline__ float lo(const QueryDev& q, int i) { return q.fbox_lo[i]; }
  static __device__ __forceinline__ float ext(const QueryDev& q, int i) { return q.fbox_ext[i]; }
  static __device__ __forceinline__ float hi(const QueryDev& q, int i) { return q.fbox_lo[i] + q.fbox_ext[i]; }
};
template <> struct BoxC<double> {
  static __device__ __forceinline__ double s(const QueryDev& q, int f) { return q.face_s[f]; }
  static __device__ __forceinline__ double lo(const QueryDev& q, int i) { return q.box_lo[i]; }
  static __device__ __forceinline__ double ext(const QueryDev& q, int i) { return q.box_hi[i] - q.box_lo[i]; }
  static __device__ __forceinline__ double hi(const QueryDev& q, int i) { return q.box_hi[i]; }
};

// Inward normal speed of the Maxwell box faces: the free-stream Maxwellian
// restricted to x = v_n / c_mp > 0 (density exp(-(x - s)^2), no flux factor),
// whose survival function erfc(x - s) / erfc(-s) = 1 - u inverts in closed
// form.  1 - u is exact for these uniforms.  A face whose erfc(-s) underflows
// carries no particle ids (its flux share is below 1e-35); the guard only
// keeps a non-finite value out of the ray set-up.
template <typename R>
__device__ __forceinline__ R truncated_normal_inverse(R u, R s) {
  R x = s + Fn<R>::erfcinv(((R)1 - u) * Fn<R>::erfc(-s));
  if (!(x > (R)0) || !(x < (R)1e30)) x = (R)1e-30;
  return x;
}

// Rectangular-CV seeding (§I, §III.A): the face owning id pid, a uniform
// point on it, the inward normal speed from the face's law, and the
// tangential components of the drifting Maxwellian (free-stream drift plus the
// same Box-Muller pair as on the sphere).
template <typename R>
__device__ __forceinline__ void seed_box(const QueryDev& q, const QC<R>& c, const float* vn_table, uint64_t pid,
                                         const uint4& w0, uint32_t w_a, R pos[3], R vel[3]) {
  int f = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) f += pid >= q.face_end[k] ? 1 : 0;
  // face axis ax; its first tangential axis (ax + 1) mod 3 takes w0.x, the second w0.y
  const int ax = f >> 1, a1 = ax == 2 ? 0 : ax + 1;
  const bool hi_face = (f & 1) == 0;
  const R s_f = BoxC<R>::s(q, f);
  const R vn = q.cv_kind == TPMC_CV_BOX_FLUX ? normal_speed_inverse<R>(uniform<R>(w0.z), s_f, vn_table)
                                             : truncated_normal_inverse<R>(uniform<R>(w0.z), s_f);
  const R rad = Fn<R>::sqrt(-Fn<R>::log(uniform<R>(w0.w)));
  R sa, ca;
  Fn<R>::sincospi((R)2 * uniform<R>(w_a), &sa, &ca);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (i == ax) {
      pos[i] = hi_face ? BoxC<R>::hi(q, i) : BoxC<R>::lo(q, i);
      vel[i] = hi_face ? -vn : vn;
    } else {
      const bool first = i == a1;
      pos[i] = BoxC<R>::lo(q, i) + uniform<R>(first ? w0.x : w0.y) * BoxC<R>::ext(q, i);
      vel[i] = c.S * c.vhat[i] + rad * (first ? ca : sa);
    }
  }
}

template <typename R>
__device__ __forceinline__ void seed_particle(const QueryDev& q, const QC<R>& c, const float* vn_table, uint64_t pid,
                                              R pos[3], R vel[3]) {
  // one Philox block: u_x, u_theta, u_vn, u_r from the top 23 bits of its
  // words, u_a (Box-Muller angle) from 23 low bits they leave unused
  const uint4 w0 = draws(q, pid, 0);
  const uint32_t w_a = ((w0.x & 0x1FFu) | ((w0.y & 0x1FFu) << 9) | ((w0.z & 0x1Fu) << 18)) << 9;
  if (q.cv_kind != TPMC_CV_SPHERE) {
    seed_box<R>(q, c, vn_table, pid, w0, w_a, pos, vel);
    return;
  }
  R cphi;
  const R x = latitude_inverse<R>(uniform<R>(w0.x), q, c, &cphi);
  R st, ct;
  Fn<R>::sincospi((R)2 * uniform<R>(w0.y), &st, &ct);
  const R vn = normal_speed_inverse<R>(uniform<R>(w0.z), c.S * x, vn_table);
  const R rad = Fn<R>::sqrt(-Fn<R>::log(uniform<R>(w0.w)));
  R sa, ca;
  Fn<R>::sincospi((R)2 * uniform<R>(w_a), &sa, &ca);
  const R vt1 = c.S * cphi + rad * ca;
  const R vt2 = rad * sa;
  // stream-frame vectors: out = (cphi ct, cphi st, -x), n = -out, t1 = (x ct, x st, cphi), t2 = (st, -ct, 0)
  const R ps[3] = {cphi * ct, cphi * st, -x};
  const R vs[3] = {-vn * cphi * ct + vt1 * x * ct + vt2 * st, -vn * cphi * st + vt1 * x * st - vt2 * ct,
                   vn * x + vt1 * cphi};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R rp = c.Rm[3 * i] * ps[0] + c.Rm[3 * i + 1] * ps[1] + c.Rm[3 * i + 2] * ps[2];
    pos[i] = c.center[i] + c.r_cv * rp;
    vel[i] = c.Rm[3 * i] * vs[0] + c.Rm[3 * i + 1] * vs[1] + c.Rm[3 * i + 2] * vs[2];
  }
}

// --------------------------------------------------- closest hit (§II.A)
template <typename R>
__device__ __forceinline__ R pick(const R v[3], int k) {
  return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]);
}

template <typename R> struct TriLoad;
template <> struct TriLoad<float> {
  static __device__ __forceinline__ uint32_t load(const MeshDev& m, uint32_t k, float A[3], float B[3], float C[3]) {
    const float4 a = __ldg(&m.tris[3 * k]), b = __ldg(&m.tris[3 * k + 1]), c = __ldg(&m.tris[3 * k + 2]);
    A[0] = a.x; A[1] = a.y; A[2] = a.z;
    B[0] = b.x; B[1] = b.y; B[2] = b.z;
    C[0] = c.x; C[1] = c.y; C[2] = c.z;
    return __float_as_uint(a.w);
  }
};
template <> struct TriLoad<double> {
  static __device__ __forceinline__ uint32_t load(const MeshDev& m, uint32_t k, double A[3], double B[3],
                                                  double C[3]) {
    const double2* p = reinterpret_cast<const double2*>(m.tris64 + 12 * (size_t)k);
    const double2 p0 = __ldg(p), p1 = __ldg(p + 1), p2 = __ldg(p + 2), p3 = __ldg(p + 3), p4 = __ldg(p + 4);
    A[0] = p0.x; A[1] = p0.y; A[2] = p1.x;
    B[0] = p1.y; B[1] = p2.x; B[2] = p2.y;
    C[0] = p3.x; C[1] = p3.y; C[2] = p4.x;
    return (uint32_t)p4.y;
  }
};

// Edge function without contraction so that a shared edge evaluates to exactly
// opposite values in its two triangles (watertightness).
__device__ __forceinline__ float edge_fn(float a, float b, float c, float d) {
  return __fsub_rn(__fmul_rn(a, b), __fmul_rn(c, d));
}
__device__ __forceinline__ double edge_fn(double a, double b, double c, double d) {
  return __dsub_rn(__dmul_rn(a, b), __dmul_rn(c, d));
}

// a b - c d in float with the sign of the exact value, and exactly 0 when
// a b = c d: Kahan's algorithm, w = c d, e = w - c d (exact by an FMA),
// f = round(a b - w), result f + e, whose relative error is at most two units
// in the last place (Jeannerod, Louvet & Muller, Math. Comp. 2013).  It
// decides the watertight test's ties in float where the plain edge function
// rounds to 0.
__device__ __forceinline__ float edge_fn_exact(float a, float b, float c, float d) {
  const float w = __fmul_rn(c, d);
  const float e = __fmaf_rn(-c, d, w);
  const float f = __fmaf_rn(a, b, -w);
  return __fadd_rn(f, e);
}

template <typename R>
struct Ray {
  R o[3], d[3], inv[3], oi[3];
  R tlo;
  // wide trees: visit position (0 first) of each child-box corner c (nibble c
  // of ptab) and the corner at each position (nibble p of stab)
  uint32_t ptab, stab;
  uint32_t nsel[3];  // binary trees: selectors of the near box planes (ray_to_grid)
};

// Woop, Benthin & Wald (JCGT 2013): shear the ray onto +z of a permuted frame.
template <typename R>
struct Shear {
  R Sx, Sy, Sz;
  int kx, ky, kz;
};

template <typename R>
__device__ __forceinline__ Shear<R> make_shear(const R d[3]) {
  Shear<R> s;
  const R ax = Fn<R>::fabs(d[0]), ay = Fn<R>::fabs(d[1]), az = Fn<R>::fabs(d[2]);
  s.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  s.kx = s.kz == 2 ? 0 : s.kz + 1;
  s.ky = s.kx == 2 ? 0 : s.kx + 1;
  if (pick(d, s.kz) < (R)0) { const int t = s.kx; s.kx = s.ky; s.ky = t; }
  s.Sz = Fn<R>::rcp(pick(d, s.kz));
  s.Sx = pick(d, s.kx) * s.Sz;
  s.Sy = pick(d, s.ky) * s.Sz;
  return s;
}

template <typename R>
__device__ __forceinline__ void make_ray(Ray<R>& r, const R o[3], const R d[3], R tlo) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.o[i] = o[i];
    r.d[i] = d[i];
    const R di = Fn<R>::fabs(d[i]) < (R)1e-30 ? copysign((R)1e-30, d[i]) : d[i];
    r.inv[i] = Fn<R>::rcp(di);
    r.oi[i] = o[i] * r.inv[i];
  }
  r.tlo = tlo;
}

// Watertight ray/triangle test; updates (tbest, best) by nearest t, then lower index.
template <typename R>
__device__ __forceinline__ void test_triangle(const Ray<R>& r, const Shear<R>& sh, const R V0[3], const R V1[3], const R V2[3],
                                              uint32_t id, R& tbest, uint32_t& best) {
  R A[3], B[3], C[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) { A[i] = V0[i] - r.o[i]; B[i] = V1[i] - r.o[i]; C[i] = V2[i] - r.o[i]; }
  const int kx = sh.kx, ky = sh.ky, kz = sh.kz;
  const R Akz = pick(A, kz), Bkz = pick(B, kz), Ckz = pick(C, kz);
  const R Ax = pick(A, kx) - sh.Sx * Akz, Ay = pick(A, ky) - sh.Sy * Akz;
  const R Bx = pick(B, kx) - sh.Sx * Bkz, By = pick(B, ky) - sh.Sy * Bkz;
  const R Cx = pick(C, kx) - sh.Sx * Ckz, Cy = pick(C, ky) - sh.Sy * Ckz;
  R U = edge_fn(Cx, By, Cy, Bx);
  R V = edge_fn(Ax, Cy, Ay, Cx);
  R W = edge_fn(Bx, Ay, By, Ax);
  if constexpr (sizeof(R) == 4) {
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
      // the ray meets an edge or a vertex to float rounding: the exact signs decide
      U = edge_fn_exact(Cx, By, Cy, Bx);
      V = edge_fn_exact(Ax, Cy, Ay, Cx);
      W = edge_fn_exact(Bx, Ay, By, Ax);
    }
  }
  if ((U < (R)0 || V < (R)0 || W < (R)0) && (U > (R)0 || V > (R)0 || W > (R)0)) return;
  R det = U + V + W;
  if (det == (R)0) return;
  R T = U * (sh.Sz * Akz) + V * (sh.Sz * Bkz) + W * (sh.Sz * Ckz);
  if (det < (R)0) { det = -det; T = -T; }
  if (T <= r.tlo * det || T > tbest * det) return;
  const R t = T * Fn<R>::rcp(det);
  if (t < tbest || (t == tbest && id < best)) { tbest = t; best = id; }
}

// Three-input min and max (one instruction each for float on sm_100 and later).
__device__ __forceinline__ float max3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ double max3(double a, double b, double c) { return fmax(fmax(a, b), c); }
__device__ __forceinline__ double min3(double a, double b, double c) { return fmin(fmin(a, b), c); }

template <typename R>
__device__ __forceinline__ void slab(R lo, R hi, R inv, R oi, R& tn, R& tf) {
  const R a = fma(lo, inv, -oi), b = fma(hi, inv, -oi);
  tn = fmin(a, b);
  tf = fmax(a, b);
}

// Binary trees keep their boxes on the mesh's grid: plane = qorigin + q qstep.
// The ray's slab constants are turned into grid units once per segment, so
// that a node's plane q, read as the float 2^23 + q (exact), gives its
// distance t = (2^23 + q) inv' - oi' in one FMA: inv' = qstep / d (exact,
// qstep is a power of two) and oi' = 2^23 inv' - (qorigin - o) / d.  The
// rounding of oi' is below half a grid step, inside the one step by which
// the builder widens every box.  A box's lo and hi along an axis share a
// word, and nsel[a] is the byte selector that reads the plane the ray meets
// first along a (lo where it runs towards +a); the other plane's selector is
// nsel[a] ^ 0x22.  The near and far distances then need no min and max.
template <typename R>
__device__ __forceinline__ void ray_to_grid(Ray<R>& r, const MeshDev& m) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R sa = (R)m.qstep[i] * r.inv[i];
    const R oa = fma((R)m.qorigin[i], r.inv[i], -r.oi[i]);
    r.inv[i] = sa;
    r.oi[i] = fma((R)8388608.0, sa, -oa);
    r.nsel[i] = sa >= (R)0 ? 0x7610u : 0x7632u;
  }
}

// A 16-bit coordinate of word w (the half that selector sel picks) as the float 2^23 + q (exact).
__device__ __forceinline__ float grid_q(uint32_t w, uint32_t sel) {
  return __int_as_float((int)__byte_perm(w, 0x4B000000u, sel));
}

// Resumable traversal of one ray, organised as in Aila & Laine's
// "while-while" scheme with speculative traversal: a warp steps through inner
// nodes until every searching lane holds a leaf, then all of them test their
// leaves together, so node visits and triangle tests run in separate, mostly
// converged loops.  A lane that found a leaf postpones it and keeps descending
// while other lanes are still searching.
constexpr int kDone = (int)0x80000000;  // no valid leaf code: first + count would exceed 2^24

// Traversal stack entry: a stacked child and its entry distance.  In float
// the pair is one 8-byte local-memory access per push and per pop (two 4-byte
// arrays took two).
template <typename R> struct StackE;
template <> struct __align__(8) StackE<float> { int node; float t; };
template <> struct __align__(16) StackE<double> { double t; int node; int pad; };
__device__ __forceinline__ void stack_put(StackE<float>* s, int i, int node, float t) {
  *reinterpret_cast<int2*>(s + i) = make_int2(node, __float_as_int(t));
}
__device__ __forceinline__ void stack_put(StackE<double>* s, int i, int node, double t) {
  s[i].t = t;
  s[i].node = node;
}
__device__ __forceinline__ void stack_get(const StackE<float>* s, int i, int& node, float& t) {
  const int2 v = *reinterpret_cast<const int2*>(s + i);
  node = v.x;
  t = __int_as_float(v.y);
}
__device__ __forceinline__ void stack_get(const StackE<double>* s, int i, int& node, double& t) {
  node = s[i].node;
  t = s[i].t;
}

template <typename R>
struct Trav {
  R tbest;
  uint32_t best;
  int cur;   // inner node >= 0; a leaf found while one is postponed (< 0); kDone when the stack is empty
  int leaf;  // postponed leaf (< 0), or 0 for none
  int sp;
};

template <typename R>
__device__ __forceinline__ void trav_begin(Trav<R>& t) {
  t.tbest = (R)CUDART_INF;
  t.best = 0xFFFFFFFFu;
  t.cur = 0;
  t.leaf = 0;
  t.sp = 0;
}

// Next stacked candidate whose entry distance is still below the best hit.
template <typename R>
__device__ __forceinline__ int trav_pop(Trav<R>& t, const StackE<R>* stack) {
  while (t.sp > 0) {
    --t.sp;
    int node;
    R te;
    stack_get(stack, t.sp, node, te);
    if (te <= t.tbest) return node;
  }
  return kDone;
}

// One inner node: test both children, continue with the nearer hit child,
// stack the farther one; the first leaf reached is postponed.  STAGE: nodes
// below n_stage come from the copy in shared memory.
template <typename R, bool STAGE>
__device__ __forceinline__ void trav_inner(const MeshDev& m, const float4* __restrict__ s_nodes, uint32_t n_stage,
                                           const Ray<R>& r, Trav<R>& t, StackE<R>* stack, uint32_t& n_nodes,
                                           int* err) {
  ++n_nodes;
  float4 n0, n1;
  if (STAGE && (uint32_t)t.cur < n_stage) {
    n0 = s_nodes[2 * t.cur]; n1 = s_nodes[2 * t.cur + 1];
  } else {
    const float4* g = m.nodes + 2 * (size_t)t.cur;
    n0 = __ldg(g); n1 = __ldg(g + 1);
  }
  // child 0: x, y, z words n0.x, n0.y, n0.z; child 1: n0.w, n1.x, n1.y; child codes n1.z, n1.w
  const uint32_t w[6] = {__float_as_uint(n0.x), __float_as_uint(n0.y), __float_as_uint(n0.z),
                         __float_as_uint(n0.w), __float_as_uint(n1.x), __float_as_uint(n1.y)};
  R tn[2][3], tf[2][3];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      tn[c][a] = fma((R)grid_q(w[3 * c + a], r.nsel[a]), r.inv[a], -r.oi[a]);
      tf[c][a] = fma((R)grid_q(w[3 * c + a], r.nsel[a] ^ 0x22u), r.inv[a], -r.oi[a]);
    }
  const R tmin0 = max3(tn[0][0], tn[0][1], fmax(tn[0][2], r.tlo));
  const R tmax0 = min3(tf[0][0], tf[0][1], fmin(tf[0][2], t.tbest));
  const R tmin1 = max3(tn[1][0], tn[1][1], fmax(tn[1][2], r.tlo));
  const R tmax1 = min3(tf[1][0], tf[1][1], fmin(tf[1][2], t.tbest));
  const bool h0 = tmin0 <= tmax0, h1 = tmin1 <= tmax1;
  int c0 = __float_as_int(n1.z), c1 = __float_as_int(n1.w);
  if (h0 && h1) {
    R tfar = tmin1;
    if (tmin1 < tmin0) { const int x = c0; c0 = c1; c1 = x; tfar = tmin0; }
    if (t.sp >= kMaxStack) {
      atomicOr(err, 1);
      t.cur = kDone;
      t.leaf = 0;
      return;
    }
    stack_put(stack, t.sp, c1, tfar);
    ++t.sp;
    t.cur = c0;
  } else if (h0) {
    t.cur = c0;
  } else if (h1) {
    t.cur = c1;
  } else {
    t.cur = trav_pop(t, stack);
  }
  if (t.cur < 0 && t.cur != kDone && t.leaf == 0) {
    t.leaf = t.cur;
    t.cur = trav_pop(t, stack);
  }
}

// The postponed leaf: test its triangles; then a leaf found meanwhile becomes
// the postponed one.  Returns true when the ray's traversal is finished.
template <typename R>
__device__ __forceinline__ bool trav_leaf(const MeshDev& m, const Ray<R>& r, uint32_t last, Trav<R>& t,
                                          const StackE<R>* stack, uint32_t& n_tris) {
  const uint32_t code = ~(uint32_t)t.leaf;
  const uint32_t first = code & 0xFFFFFFu, count = code >> 24;
  const Shear<R> sh = make_shear<R>(r.d);
  for (uint32_t k = first; k < first + count; ++k) {
    R V0[3], V1[3], V2[3];
    const uint32_t id = TriLoad<R>::load(m, k, V0, V1, V2);
    if (id == last) continue;
    ++n_tris;
    test_triangle<R>(r, sh, V0, V1, V2, id, t.tbest, t.best);
  }
  t.leaf = 0;
  if (t.cur < 0 && t.cur != kDone) {
    t.leaf = t.cur;
    t.cur = trav_pop(t, stack);
  }
  return t.leaf == 0 && t.cur == kDone;
}

// ------------------------------------- compressed wide BVH traversal
// The children of a wide node are visited in the order of their slots'
// corners (bit a of a corner: the child lies towards +a) as seen along the
// ray: the corner's bits are flipped on the axes where the ray runs towards
// -a, then read most significant first along the ray's dominant axis, next
// the second, last the third.  A near child thus comes before a far one
// along the axis that matters most, with no sort.  ptab holds each slot's
// visit position (nibble s), stab the slot at each position (nibble p).
template <int W, typename R>
__device__ __forceinline__ void ray_order(Ray<R>& r) {
  const R ax = Fn<R>::fabs(r.d[0]), ay = Fn<R>::fabs(r.d[1]), az = Fn<R>::fabs(r.d[2]);
  const uint32_t flip = (r.d[0] < (R)0 ? 1u : 0u) | (r.d[1] < (R)0 ? 2u : 0u) | (r.d[2] < (R)0 ? 4u : 0u);
  // axes by decreasing |d|
  uint32_t a0 = 0, a1 = 1, a2 = 2;
  {
    R v0 = ax, v1 = ay, v2 = az;
    if (v1 > v0) { const R t = v0; v0 = v1; v1 = t; const uint32_t u = a0; a0 = a1; a1 = u; }
    if (v2 > v1) { const R t = v1; v1 = v2; v2 = t; const uint32_t u = a1; a1 = a2; a2 = u; }
    if (v1 > v0) { const uint32_t u = a0; a0 = a1; a1 = u; }
  }
  uint32_t ptab = 0, stab = 0;
#pragma unroll
  for (uint32_t slot = 0; slot < (uint32_t)W; ++slot) {
    // the slot's corner (kWide4Corner for 4-wide nodes)
    const uint32_t c = W == 8 ? slot : (slot == 0 ? 0u : (slot == 1 ? 3u : (slot == 2 ? 5u : 6u)));
    const uint32_t t = c ^ flip;
    const uint32_t pos = (((t >> a0) & 1u) << 2) | (((t >> a1) & 1u) << 1) | ((t >> a2) & 1u);
    ptab |= pos << (4 * slot);
    stab |= slot << (4 * pos);
  }
  r.ptab = ptab;
  r.stab = stab;
}

// Traversal state of one ray in a wide tree.
//   gx, gy: the current node group, the hit inner children of one node still
//           to visit: gx = child_base | (hit positions << 24), gy = (lower
//           bound on their entry distances, low 8 bits cleared) | imask;
//   tb, tm: triangles to test: tb + k for every bit k of tm.
// A stack entry is a node group (gx, gy), or a postponed triangle group
// (tm, tb | 2^31): a node group's gy is a positive float's bits, bit 31 clear.
template <typename R>
struct TravW {
  R tbest;
  uint32_t best;
  uint32_t gx, gy, tb, tm;
  int sp;
};

constexpr uint32_t kTriEntry = 0x80000000u;

template <typename R>
__device__ __forceinline__ void travw_begin(TravW<R>& t, const Ray<R>& r) {
  t.tbest = (R)CUDART_INF;
  t.best = 0xFFFFFFFFu;
  t.gx = (1u << (r.ptab & 7u)) << 24;  // the root: an inner child in slot 0 of node base 0
  t.gy = 1u;
  t.tb = 0;
  t.tm = 0;
  t.sp = 0;
}

// Next stacked work: a node group whose entry bound is still within the best
// hit becomes the current group; a postponed triangle group becomes the
// triangle mask (only taken when the mask is empty).
template <typename R>
__device__ __forceinline__ void travw_pop(TravW<R>& t, const uint2* stack) {
  while (t.sp > 0) {
    --t.sp;
    const uint2 e = stack[t.sp];
    if (e.y & kTriEntry) {
      t.tm = e.x;
      t.tb = e.y & ~kTriEntry;
      return;
    }
    if ((R)__uint_as_float(e.y & ~0xFFu) <= t.tbest) {
      t.gx = e.x;
      t.gy = e.y;
      return;
    }
  }
}

// Byte k of w as a float, exactly: 2^23 + b built in the bits, then 2^23 taken off.
__device__ __forceinline__ float byte_float(uint32_t w, uint32_t k) {
  return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7440u + k)) - 8388608.0f;
}


// Float bound below t (its low 8 bits are cleared to make room for imask).
__device__ __forceinline__ uint32_t t_bits_down(float t) { return __float_as_uint(t) & ~0xFFu; }
__device__ __forceinline__ uint32_t t_bits_down(double t) { return __float_as_uint(__double2float_rd(t)) & ~0xFFu; }

// One node of the group: the next hit child in visit order is fetched and its
// W child boxes tested; the group's other children are stacked.  The hit
// inner children form the new group; the hit leaves' triangles become the
// triangle mask, or, when the lane still holds one (speculative descent),
// a postponed group on the stack.
template <typename R, int W>
__device__ __forceinline__ void travw_node(const MeshDev& m, const Ray<R>& r, TravW<R>& t, uint2* stack,
                                           uint32_t& n_nodes, int* err) {
  constexpr int F4 = W == 8 ? 5 : 4;
  const uint32_t hits = t.gx >> 24;
  const uint32_t pos = __ffs(hits) - 1;
  const uint32_t rest = hits & (hits - 1u);
  const uint32_t slot = (r.stab >> (4 * pos)) & 7u;
  const uint32_t node = (t.gx & 0xFFFFFFu) + __popc(t.gy & 0xFFu & ((1u << slot) - 1u));
  if (rest != 0u) {
    if (t.sp >= kMaxStackW) {
      atomicOr(err, 1);
      t.gx = 0;
      t.tm = 0;
      t.sp = 0;
      return;
    }
    stack[t.sp] = make_uint2((t.gx & 0xFFFFFFu) | (rest << 24), t.gy);
    ++t.sp;
  }
  ++n_nodes;
  float4 v[F4];
  const float4* g = m.nodes + (size_t)F4 * node;
#pragma unroll
  for (int i = 0; i < F4; ++i) v[i] = __ldg(g + i);
  const uint32_t ew = __float_as_uint(v[0].w);
  const uint32_t imask = ew >> 24;
  // per axis: grid step times 1/d, and the grid origin's distance
  R sa[3], oa[3];
  const float p[3] = {v[0].x, v[0].y, v[0].z};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    sa[a] = (R)__uint_as_float(((ew >> (8 * a)) & 0xFFu) << 23) * r.inv[a];
    oa[a] = fma((R)p[a], r.inv[a], -r.oi[a]);
  }
  // plane words (W = 8: two per plane, slots 0-3 then 4-7; W = 4: one per plane)
  constexpr int PP = W == 8 ? 2 : 1;
  uint32_t q[6 * PP];
#pragma unroll
  for (int i = 0; i < 6 * PP; ++i) {
    const float4& f = v[2 + i / 4];
    q[i] = __float_as_uint((i & 3) == 0 ? f.x : ((i & 3) == 1 ? f.y : ((i & 3) == 2 ? f.z : f.w)));
  }
  // near and far planes along each axis: lo first where the ray runs towards +a
  uint32_t qn[3][PP], qf[3][PP];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const bool pos_dir = r.inv[a] >= (R)0;
#pragma unroll
    for (int h = 0; h < PP; ++h) {
      const uint32_t lo = q[PP * a + h], hi = q[PP * (a + 3) + h];
      qn[a][h] = pos_dir ? lo : hi;
      qf[a][h] = pos_dir ? hi : lo;
    }
  }
  uint32_t hitbits = 0;
  R tmin_hit = (R)CUDART_INF;
#pragma unroll
  for (int s = 0; s < W; ++s) {
    const int h = s >> 2, k = s & 3;
    const R tn = max3(max3(fma((R)byte_float(qn[0][h], k), sa[0], oa[0]), fma((R)byte_float(qn[1][h], k), sa[1], oa[1]),
                           fma((R)byte_float(qn[2][h], k), sa[2], oa[2])), r.tlo, r.tlo);
    const R tf = min3(fma((R)byte_float(qf[0][h], k), sa[0], oa[0]), fma((R)byte_float(qf[1][h], k), sa[1], oa[1]),
                      min3(fma((R)byte_float(qf[2][h], k), sa[2], oa[2]), t.tbest, t.tbest));
    const bool hit = tn <= tf;
    hitbits |= hit ? (1u << s) : 0u;
    tmin_hit = fmin(tmin_hit, hit ? tn : (R)CUDART_INF);
  }
  // hit inner children by visit position; hit leaves' triangles
  uint32_t inner = hitbits & imask, new_hits = 0;
  while (inner != 0u) {
    const uint32_t s = __ffs(inner) - 1;
    inner &= inner - 1u;
    new_hits |= 1u << ((r.ptab >> (4 * s)) & 7u);
  }
  uint32_t leaves = hitbits & ~imask, tris = 0;
  const uint32_t meta0 = __float_as_uint(v[1].z), meta1 = __float_as_uint(v[1].w);
  while (leaves != 0u) {
    const uint32_t s = __ffs(leaves) - 1;
    leaves &= leaves - 1u;
    const uint32_t meta = ((s < 4 ? meta0 : meta1) >> (8 * (s & 3u))) & 0xFFu;
    tris |= (0xFu >> (3u - (meta >> 5))) << (meta & 31u);
  }
  t.gx = __float_as_uint(v[1].x) | (new_hits << 24);
  t.gy = t_bits_down(tmin_hit) | imask;
  if (tris != 0u) {
    if (t.tm == 0u) {
      t.tb = __float_as_uint(v[1].y);
      t.tm = tris;
    } else if (t.sp < kMaxStackW) {  // speculative step: postpone these triangles
      stack[t.sp] = make_uint2(tris, __float_as_uint(v[1].y) | kTriEntry);
      ++t.sp;
    } else {
      atomicOr(err, 1);
      t.gx = 0;
      t.tm = 0;
      t.sp = 0;
    }
  }
}

// Triangles of the mask (a node's hit leaves), in any order: nearest t wins.
template <typename R>
__device__ __forceinline__ void travw_tris(const MeshDev& m, const Ray<R>& r, uint32_t last, TravW<R>& t,
                                           uint32_t& n_tris) {
  const Shear<R> sh = make_shear<R>(r.d);
  while (t.tm != 0u) {
    const uint32_t k = __ffs(t.tm) - 1;
    t.tm &= t.tm - 1u;
    R V0[3], V1[3], V2[3];
    const uint32_t id = TriLoad<R>::load(m, t.tb + k, V0, V1, V2);
    if (id == last) continue;
    ++n_tris;
    test_triangle<R>(r, sh, V0, V1, V2, id, t.tbest, t.best);
  }
}

// ------------------------------------------------ re-emission (§II.A)
template <typename R> struct Frame;
// A triangle's frame, and its exposed sides (bit 0: the side n points to,
// bit 1: the other): sides that the whole mesh lies behind.
template <> struct Frame<float> {
  static __device__ __forceinline__ uint32_t load(const MeshDev& m, uint32_t id, float n[3], float t1[3]) {
    const float4 a = __ldg(&m.frames[2 * id]), b = __ldg(&m.frames[2 * id + 1]);
    n[0] = a.x; n[1] = a.y; n[2] = a.z;
    t1[0] = b.x; t1[1] = b.y; t1[2] = b.z;
    return __float_as_uint(b.w);
  }
};
template <> struct Frame<double> {
  static __device__ __forceinline__ uint32_t load(const MeshDev& m, uint32_t id, double n[3], double t1[3]) {
    const double* f = m.frames64 + 8 * (size_t)id;
    n[0] = __ldg(f); n[1] = __ldg(f + 1); n[2] = __ldg(f + 2);
    t1[0] = __ldg(f + 4); t1[1] = __ldg(f + 5); t1[2] = __ldg(f + 6);
    return (uint32_t)__ldg(f + 7);
  }
};

// Maxwell model: with probability eps diffuse re-emission from the
// flux-weighted half-range Maxwellian at T_W about the hit-side normal
// (normal speed c_W sqrt(-ln u1), tangential c_W sqrt(-ln u2) at angle 2 pi u3
// in the frame (t1, n x t1)); otherwise specular reflection.
template <typename R> struct CllC;
template <> struct CllC<float> {
  static __device__ __forceinline__ float get(const QueryDev& q, int k) { return q.fcll[k]; }
};
template <> struct CllC<double> {
  static __device__ __forceinline__ double get(const QueryDev& q, int k) { return q.cll[k]; }
};

// Cercignani-Lampis-Lord re-emission (Lord's sampling of the CL kernel), in
// units of c_W about the hit-side normal n_out (sgn n): with the incident
// normal speed v_n and tangential components (v_t1, v_t2) along (t1, n x t1),
//   r = sqrt(-alpha_n ln u0), theta = 2 pi u1,
//   v_n' = sqrt(r^2 + (1 - alpha_n) v_n^2 + 2 r sqrt(1 - alpha_n) v_n cos theta),
//   rho = sqrt(-alpha_t ln u2), phi = 2 pi u3,
//   v_t' = sqrt(1 - alpha_t) v_t + rho (cos phi, sin phi).
template <typename R>
__device__ __forceinline__ void reemit_cll(const QueryDev& q, R cw, const uint4& w, R sgn, const R n[3],
                                           const R t1[3], R v[3]) {
  const R t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
  const R inv_cw = (R)1 / cw;
  const R vn = -sgn * (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) * inv_cw;
  const R vt1 = (v[0] * t1[0] + v[1] * t1[1] + v[2] * t1[2]) * inv_cw;
  const R vt2 = (v[0] * t2[0] + v[1] * t2[1] + v[2] * t2[2]) * inv_cw;
  const R r = Fn<R>::sqrt(-CllC<R>::get(q, 0) * Fn<R>::log(uniform<R>(w.x)));
  R st, ct;
  Fn<R>::sincospi((R)2 * uniform<R>(w.y), &st, &ct);
  const R b = CllC<R>::get(q, 1) * vn;
  const R vn_out = Fn<R>::sqrt(fmax(r * r + b * b + (R)2 * r * b * ct, (R)0));
  const R rho = Fn<R>::sqrt(-CllC<R>::get(q, 2) * Fn<R>::log(uniform<R>(w.z)));
  R sp, cp;
  Fn<R>::sincospi((R)2 * uniform<R>(w.w), &sp, &cp);
  const R a1 = CllC<R>::get(q, 3) * vt1 + rho * cp, a2 = CllC<R>::get(q, 3) * vt2 + rho * sp;
#pragma unroll
  for (int i = 0; i < 3; ++i) v[i] = cw * (sgn * vn_out * n[i] + a1 * t1[i] + a2 * t2[i]);
}

// CLL: compiled into the kernel variants that serve launches holding a CLL query.
template <typename R, bool CLL>
__device__ __forceinline__ void reemit(const QueryDev& q, R cw, uint64_t pid, uint32_t bounce, const R n[3],
                                       const R t1[3], R v[3]) {
  const uint4 w = draws(q, pid, 2 + bounce);
  const R vdn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
  if constexpr (CLL) {
    if (q.gsi_model == TPMC_GSI_CLL) {
      reemit_cll<R>(q, cw, w, vdn < (R)0 ? (R)1 : (R)-1, n, t1, v);
      return;
    }
  }
  if ((w.x >> 9) < q.eps_k) {  // u < eps, decided on the integer behind u
    const R sgn = vdn < (R)0 ? (R)1 : (R)-1;
    const R vn = cw * Fn<R>::sqrt(-Fn<R>::log(uniform<R>(w.y)));
    const R vt = cw * Fn<R>::sqrt(-Fn<R>::log(uniform<R>(w.z)));
    R s, co;
    Fn<R>::sincospi((R)2 * uniform<R>(w.w), &s, &co);
    const R t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = sgn * vn * n[i] + vt * (co * t1[i] + s * t2[i]);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = v[i] - (R)2 * vdn * n[i];
  }
}

__device__ __forceinline__ long long quantize(float x) { return __float2ll_rn(x); }
__device__ __forceinline__ long long quantize(double x) { return __double2ll_rn(x); }

// Per-lane partial sums for the query the lane is working on.  They live in
// shared memory (one slot per thread), which keeps them out of the registers
// the traversal needs.
// d2lo and d2hi hold the lane's sum of squared drag contributions as the
// 96-bit integer d2hi 2^64 + d2lo (units of the query's quantum2).
struct LaneAcc {
  long long F[3], T[3];
  unsigned long long d2lo;
  uint32_t hits, hit_particles, truncated, particles;
  int q;
  uint32_t d2hi;
  // the lane's particle: its id (bits 0-39) and the hits so far (bits 40-63),
  // kept here rather than in registers the traversal loop needs
  unsigned long long pb;
};

__device__ __forceinline__ void lane_reset(LaneAcc& a, int q) {
#pragma unroll
  for (int i = 0; i < 3; ++i) { a.F[i] = 0; a.T[i] = 0; }
  a.hits = a.hit_particles = a.truncated = a.particles = 0;
  a.d2lo = 0;
  a.d2hi = 0;
  a.q = q;
}

// Adds one particle's squared drag contribution d^2 (c_mp^2 units), rounded to
// the query's quantum2; the set-up bounds every particle's term below 2^62.
__device__ __forceinline__ unsigned long long quantize_sq(float x) { return __float2ull_rn(x); }
__device__ __forceinline__ unsigned long long quantize_sq(double x) { return __double2ull_rn(x); }
__device__ __forceinline__ void lane_add_d2(LaneAcc& a, unsigned long long x) {
  const unsigned long long lo = a.d2lo + x;
  a.d2hi += lo < x ? 1u : 0u;
  a.d2lo = lo;
}

// Adds the 96-bit sum hi 2^64 + lo of one flush to the three limbs of the
// stripe's squared-drag sum: bits 0-29, bits 30-59, and hi 2^4 + (lo >> 60).
// Every flush carries at least one particle and a query has at most 2^34, so
// each low limb stays below 2^34 2^30 = 2^64; the top limb stays below the
// exact total over 2^60, which is below 2^36 (each particle's term is below
// 2^62).
__device__ __forceinline__ void add_d2(AccStripe& A, unsigned long long lo, unsigned long long hi) {
  constexpr unsigned long long kM30 = (1ull << 30) - 1ull;
  const unsigned long long l0 = lo & kM30, l1 = (lo >> 30) & kM30, l2 = (hi << 4) | (lo >> 60);
  if (l0) atomicAdd(&A.d2[0], l0);
  if (l1) atomicAdd(&A.d2[1], l1);
  if (l2) atomicAdd(&A.d2[2], l2);
}

// The stripe of a query's sums that this warp adds to.
__device__ __forceinline__ int acc_stripe() {
  return (int)((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) & (unsigned)(kAccStripes - 1));
}

__device__ __forceinline__ void lane_flush(AccStripe* acc, uint32_t stride, LaneAcc& a, int stripe) {
  if (a.q < 0 || a.particles == 0) return;
  AccStripe& A = acc[(size_t)stripe * stride + a.q];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (a.F[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&A.F[i]), (unsigned long long)a.F[i]);
    if (a.T[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&A.T[i]), (unsigned long long)a.T[i]);
  }
  if (a.hits) atomicAdd(&A.hits, (unsigned long long)a.hits);
  if (a.hit_particles) atomicAdd(&A.hit_particles, (unsigned long long)a.hit_particles);
  if (a.truncated) atomicAdd(&A.truncated, (unsigned long long)a.truncated);
  atomicAdd(&A.particles, (unsigned long long)a.particles);
  add_d2(A, a.d2lo, a.d2hi);
}

// Flush at the end of the kernel, where every lane of the warp arrives
// together (the main loop ends on a warp-uniform test).  When all lanes hold
// sums of the same query, the warp adds them by a butterfly of shuffles (the
// 128-bit sum of squares with its carry) and one lane issues the atomics;
// lanes of mixed queries flush one by one.  Integer sums, so the result is
// the same either way.
__device__ __forceinline__ void warp_flush(AccStripe* acc, uint32_t stride, LaneAcc& a, int stripe) {
  const unsigned same = __match_any_sync(kFull, a.q);
  if (same != kFull || a.q < 0) {
    lane_flush(acc, stride, a, stripe);
    return;
  }
  long long F[3], T[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) { F[i] = a.F[i]; T[i] = a.T[i]; }
  unsigned long long lo = a.d2lo, hi = a.d2hi;
  unsigned long long hits = a.hits, hitp = a.hit_particles, trunc = a.truncated, parts = a.particles;
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      F[i] += __shfl_xor_sync(kFull, F[i], m);
      T[i] += __shfl_xor_sync(kFull, T[i], m);
    }
    const unsigned long long olo = __shfl_xor_sync(kFull, lo, m), ohi = __shfl_xor_sync(kFull, hi, m);
    const unsigned long long nlo = lo + olo;
    hi += ohi + (nlo < lo ? 1ull : 0ull);
    lo = nlo;
    hits += __shfl_xor_sync(kFull, hits, m);
    hitp += __shfl_xor_sync(kFull, hitp, m);
    trunc += __shfl_xor_sync(kFull, trunc, m);
    parts += __shfl_xor_sync(kFull, parts, m);
  }
  if ((threadIdx.x & 31u) != 0u || parts == 0) return;
  AccStripe& A = acc[(size_t)stripe * stride + a.q];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (F[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&A.F[i]), (unsigned long long)F[i]);
    if (T[i]) atomicAdd(reinterpret_cast<unsigned long long*>(&A.T[i]), (unsigned long long)T[i]);
  }
  if (hits) atomicAdd(&A.hits, hits);
  if (hitp) atomicAdd(&A.hit_particles, hitp);
  if (trunc) atomicAdd(&A.truncated, trunc);
  atomicAdd(&A.particles, parts);
  add_d2(A, lo, hi);
}

__device__ __forceinline__ void work_flush(AccStripe* acc, uint32_t stride, int q, uint32_t n_nodes, uint32_t n_tris,
                                           int stripe) {
  if (q < 0) return;
  AccStripe& A = acc[(size_t)stripe * stride + q];
  if (n_nodes) atomicAdd(&A.nodes, (unsigned long long)n_nodes);
  if (n_tris) atomicAdd(&A.tris, (unsigned long long)n_tris);
}

// Work index g -> item (binary search over item starts).
__device__ __forceinline__ uint32_t find_item(const ItemDev* items, uint32_t n_items, uint64_t g) {
  uint32_t lo = 0, hi = n_items;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(&items[mid].g_begin) <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Per-query constants of the traced (not seeded) part, in the path's precision.
template <typename R> struct HitConst;
template <> struct HitConst<float> {
  static __device__ __forceinline__ float cw(const QueryDev& q) { return q.fc[kFcCw]; }
  static __device__ __forceinline__ float scale(const QueryDev& q) { return q.fc[kFcScale]; }
  static __device__ __forceinline__ float ref(const QueryDev& q, int i) { return q.fc[kFcRef + i]; }
  static __device__ __forceinline__ float vhat(const QueryDev& q, int i) { return q.fc[kFcVhat + i]; }
  static __device__ __forceinline__ float scale2(const QueryDev& q) { return q.fc[kFcScale2]; }
};
template <> struct HitConst<double> {
  static __device__ __forceinline__ double cw(const QueryDev& q) { return q.cw; }
  static __device__ __forceinline__ double scale(const QueryDev& q) { return 1.0 / q.quantum; }
  static __device__ __forceinline__ double ref(const QueryDev& q, int i) { return q.ref[i]; }
  static __device__ __forceinline__ double vhat(const QueryDev& q, int i) { return q.vhat[i]; }
  static __device__ __forceinline__ double scale2(const QueryDev& q) { return 1.0 / q.quantum2; }
};

// A seeded particle waiting in its warp's queue (shared memory).
template <typename R>
struct alignas(sizeof(R) == 4 ? 16 : 8) Seeded {
  R pos[3], vel[3];
  uint64_t pq;  // particle id in bits 0-39, query slot above
};
static_assert(sizeof(Seeded<float>) == 32, "a float queue slot is two 16-byte vectors");

// Float slots are written and read as two 16-byte vectors: eight lanes'
// 16-byte accesses at a 32-byte stride take two shared-memory wavefronts,
// where 4-byte fields at that stride would conflict eight ways.
template <typename R>
__device__ __forceinline__ void slot_store(Seeded<R>& e, const R pos[3], const R vel[3], uint64_t pq) {
  if constexpr (sizeof(R) == 4) {
    float4* v = reinterpret_cast<float4*>(&e);
    v[0] = make_float4(pos[0], pos[1], pos[2], vel[0]);
    v[1] = make_float4(vel[1], vel[2], __uint_as_float((uint32_t)pq), __uint_as_float((uint32_t)(pq >> 32)));
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) { e.pos[i] = pos[i]; e.vel[i] = vel[i]; }
    e.pq = pq;
  }
}

template <typename R>
__device__ __forceinline__ uint64_t slot_load(const Seeded<R>& e, R pos[3], R vel[3]) {
  if constexpr (sizeof(R) == 4) {
    const float4* v = reinterpret_cast<const float4*>(&e);
    const float4 a = v[0], b = v[1];
    pos[0] = a.x; pos[1] = a.y; pos[2] = a.z;
    vel[0] = a.w; vel[1] = b.x; vel[2] = b.y;
    return (uint64_t)__float_as_uint(b.z) | ((uint64_t)__float_as_uint(b.w) << 32);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) { pos[i] = e.pos[i]; vel[i] = e.vel[i]; }
    return e.pq;
  }
}

// Seeds particle pid of query qi into a queue slot.  Kept out of line: the
// seeding temporaries then do not stay live across the traversal loop.
template <typename R>
__device__ __noinline__ void seed_into(const TraceArgs& a, uint32_t qi, uint64_t pid, Seeded<R>& e) {
  const QueryDev& q = a.queries[qi];
  QC<R> c;
  c.load(q);
  R pos[3], vel[3];
  seed_particle<R>(q, c, a.vn_table, pid, pos, vel);
  slot_store<R>(e, pos, vel, pid | ((uint64_t)qi << kSlotPidBits));
  if (a.rec.pos != nullptr) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a.rec.pos[3 * pid + i] = (double)pos[i];
      a.rec.vel[3 * pid + i] = (double)vel[i];
    }
  }
}

constexpr uint32_t kQueue = 64;     // queue slots per warp (two seeding batches)

// Whether the ray meets the mesh's padded root box beyond tlo (the slab
// arithmetic of the node test, so a ray rejected here misses every node).
template <typename R>
__device__ __forceinline__ bool ray_meets_box(const Ray<R>& r, const MeshDev& m) {
  R tn = r.tlo, tf = (R)CUDART_INF;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R a, b;
    slab<R>((R)m.box_lo[i], (R)m.box_hi[i], r.inv[i], r.oi[i], a, b);
    tn = fmax(tn, a);
    tf = fmin(tf, b);
  }
  return tn <= tf;
}

// --------------------------------------------------------- trace kernel
// Persistent kernel.  Each warp keeps a queue of seeded particles in shared
// memory; when its lanes need particles and the queue runs low, all 32 lanes
// seed one particle each (so the inverse-CDF solves run at full warp width).
// Lanes then trace in rounds of resumable traversal steps; a round ends when
// refill_at lanes have finished their rays, and those lanes re-emit (next
// bounce) or finish their particle and take the next one from the queue.
// MINB > 0: a register-capped instantiation for 128-thread blocks with at
// least MINB resident blocks per SM (more warps to hide latency, at the cost
// of spills inside the out-of-line seeding).  MINB = 0: 256-thread blocks,
// two per SM in float (at most 128 registers), one in double.
template <int W, typename R, typename TV>
__device__ __forceinline__ void begin_trav(Ray<R>& r, TV& tv, const MeshDev& m) {
  if constexpr (W > 2) {
    ray_order<W>(r);
    travw_begin(tv, r);
  } else {
    ray_to_grid<R>(r, m);
    trav_begin(tv);
  }
}

template <typename R, int MINB, bool CLL, int W, bool COUNT>
__global__ void __launch_bounds__(MINB > 0 ? 128 : 256, MINB > 0 ? MINB : (sizeof(R) == 4 ? 2 : 1))
    trace_kernel(TraceArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr uint32_t kNodeF4 = kBinaryNodeF4;  // float4 per binary node
  // only the binary traversal reads staged nodes
  const uint32_t n_stage = W > 2 ? 0u : min(a.smem_nodes, a.mesh.n_nodes);
  float4* s_nodes = reinterpret_cast<float4*>(smem);
  if constexpr (W == 2)
    for (uint32_t i = threadIdx.x; i < kNodeF4 * n_stage; i += blockDim.x) s_nodes[i] = __ldg(&a.mesh.nodes[i]);
  Seeded<R>* queue = reinterpret_cast<Seeded<R>*>(smem + (size_t)n_stage * kNodeF4 * sizeof(float4)) +
                     (threadIdx.x >> 5) * kQueue;
  LaneAcc& acc = reinterpret_cast<LaneAcc*>(smem + (size_t)n_stage * kNodeF4 * sizeof(float4) +
                                            (size_t)(blockDim.x >> 5) * kQueue * sizeof(Seeded<R>))[threadIdx.x];
  lane_reset(acc, -1);
  __syncthreads();

  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;

  // warp-uniform state: queue ring, work pool
  uint32_t q_head = 0, q_count = 0;
  uint64_t pool_base = 0;
  uint32_t pool_rem = 0;
  bool drained = false;
  // lane's cached work item (for seeding)
  uint64_t it_g1 = 0, it_off = 0;  // cached item: end of its work range, pid - g
  uint32_t it_q = 0;

  // lane's particle
  bool has = false, tdone = true;
  int qi = -1;
  uint32_t last = 0xFFFFFFFFu;
  R dvp[3] = {0, 0, 0};  // the particle's summed momentum change (records only)
  R dpart = 0;           // its drag component, summed over its hits (for sigma)
  Ray<R> ray;
  using TV = std::conditional_t<(W > 2), TravW<R>, Trav<R>>;
  using SE = std::conditional_t<(W > 2), uint2, StackE<R>>;
  TV tv{};
  SE stack[W > 2 ? kMaxStackW : kMaxStack];
  uint32_t n_nodes = 0, n_tris = 0;

  for (;;) {
    // ---- 1. lanes whose ray is finished: re-emit, or finish the particle
    if (has && tdone) {
      const QueryDev& q = a.queries[qi];
      const uint64_t pid = acc.pb & ((1ull << kSlotPidBits) - 1);
      uint32_t bounce = (uint32_t)(acc.pb >> kSlotPidBits);
      bool finish = true;
      if (tv.best != 0xFFFFFFFFu) {
        const uint32_t hit = tv.best;
        R nrm[3], t1[3], hp[3], v_in[3];
        const uint32_t exposed = Frame<R>::load(a.mesh, hit, nrm, t1);
#pragma unroll
        for (int i = 0; i < 3; ++i) { hp[i] = ray.o[i] + tv.tbest * ray.d[i]; v_in[i] = ray.d[i]; }
        R v[3] = {ray.d[0], ray.d[1], ray.d[2]};
        reemit<R, CLL>(q, HitConst<R>::cw(q), pid, bounce, nrm, t1, v);
        R dv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          dv[i] = v_in[i] - v[i];
          if constexpr (COUNT) dvp[i] += dv[i];
        }
        dpart += dv[0] * HitConst<R>::vhat(q, 0) + dv[1] * HitConst<R>::vhat(q, 1) + dv[2] * HitConst<R>::vhat(q, 2);
        const R r0 = hp[0] - HitConst<R>::ref(q, 0), r1 = hp[1] - HitConst<R>::ref(q, 1),
                r2 = hp[2] - HitConst<R>::ref(q, 2);
        const R tq[3] = {r1 * dv[2] - r2 * dv[1], r2 * dv[0] - r0 * dv[2], r0 * dv[1] - r1 * dv[0]};
        const R sc = HitConst<R>::scale(q);
        long long qf[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          qf[i] = quantize(dv[i] * sc);
          acc.F[i] += qf[i];
          acc.T[i] += quantize(tq[i] * sc);
        }
        long long* panel = q.panel;
        if (panel != nullptr) {
          long long* pp = panel + 3 * (size_t)hit;
#pragma unroll
          for (int i = 0; i < 3; ++i)
            if (qf[i]) atomicAdd(reinterpret_cast<unsigned long long*>(pp + i), (unsigned long long)qf[i]);
        }
        if constexpr (COUNT)
          if (a.rec.tri != nullptr && bounce < a.rec.K) a.rec.tri[(size_t)pid * a.rec.K + bounce] = hit;
        ++acc.hits;
        if (bounce == 0) ++acc.hit_particles;
        ++bounce;
        acc.pb += 1ull << kSlotPidBits;
        last = hit;
        if (bounce >= q.max_bounces) {
          ++acc.truncated;
        } else {
          // The particle leaves from the side it arrived on.  When the whole
          // mesh lies behind that side (to 1e-12 m) and it leaves at more than
          // 0.01 in cos from the plane, nothing lies ahead of it beyond 1e-10 m,
          // inside the shortest hit distance: it is done, without a traversal.
          const R vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
          const R vn = v[0] * nrm[0] + v[1] * nrm[1] + v[2] * nrm[2];
          const bool escapes = (exposed & (vn > (R)0 ? 1u : 2u)) != 0u && vn * vn > (R)1e-4 * vv;
          if (!escapes) {
            // the shortest hit distance, 1e-6 m (1e-9 m in double) over the speed
            make_ray<R>(ray, hp, v, (sizeof(R) == 4 ? (R)1e-6 : (R)1e-9) * Fn<R>::rsqrt(vv));
            begin_trav<W>(ray, tv, a.mesh);
            tdone = a.mesh.n_nodes == 0;
            finish = false;
          }
        }
      }
      if (finish) {
        if (dpart != (R)0) lane_add_d2(acc, quantize_sq(dpart * dpart * HitConst<R>::scale2(q)));
        ++acc.particles;
        if (COUNT && a.rec.n_hits != nullptr) {
          a.rec.n_hits[pid] = bounce;
          a.rec.truncated[pid] = (tv.best != 0xFFFFFFFFu && bounce >= q.max_bounces) ? 1u : 0u;
#pragma unroll
          for (int i = 0; i < 3; ++i) a.rec.dv[3 * pid + i] = (double)dvp[i];
        }
        has = false;
      }
    }

    // ---- 2. idle lanes take particles from the queue; seed a batch when it runs low.
    // A particle whose ray misses the mesh's root box is counted at once (its
    // sums are zero) and the lane takes another, up to three times.
    for (int pass = 0; pass < 3; ++pass) {
      const unsigned need = __ballot_sync(kFull, !has);
      if (need == 0u) break;
      const uint32_t n_need = __popc(need);
      if (q_count < n_need && !drained && q_count + 32u <= kQueue) {
        if (pool_rem == 0) {
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(a.counter, (unsigned long long)a.chunk);
          base = __shfl_sync(kFull, base, 0);
          if (base >= a.total) {
            drained = true;
          } else {
            pool_base = base;
            const uint64_t left = a.total - base;
            pool_rem = left < (uint64_t)a.chunk ? (uint32_t)left : a.chunk;
          }
        }
        if (!drained) {
          const uint32_t nb = min(32u, pool_rem);
          if (lane < nb) {
            const uint64_t g = pool_base + lane;
            if (g >= it_g1) {  // a lane's work indices only grow
              const ItemDev item = a.items[find_item(a.items, a.n_items, g)];
              it_g1 = item.g_begin + item.count;
              it_off = item.pid_begin - item.g_begin;
              it_q = item.query;
            }
            seed_into<R>(a, it_q, g + it_off, queue[(q_head + q_count + lane) & (kQueue - 1)]);
          }
          pool_base += nb;
          pool_rem -= nb;
          q_count += nb;
        }
        __syncwarp();
      }
      const uint32_t take = min(n_need, q_count);
      const uint32_t rank = __popc(need & lt_mask);
      if (((need >> lane) & 1u) && rank < take) {
        R pos[3], vel[3];
        const uint64_t pq = slot_load<R>(queue[(q_head + rank) & (kQueue - 1)], pos, vel);
        const uint64_t pid = pq & ((1ull << kSlotPidBits) - 1);
        const int nq = (int)(pq >> kSlotPidBits);
        if (nq != acc.q) {
          if constexpr (COUNT) {
            work_flush(a.acc, a.acc_stride, acc.q, n_nodes, n_tris, acc_stripe());
            n_nodes = n_tris = 0;
          }
          lane_flush(a.acc, a.acc_stride, acc, acc_stripe());
          lane_reset(acc, nq);
        }
        qi = nq;
        make_ray<R>(ray, pos, vel,
                    (sizeof(R) == 4 ? (R)1e-6 : (R)1e-9) *
                        Fn<R>::rsqrt(vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]));
        begin_trav<W>(ray, tv, a.mesh);
        tdone = a.mesh.n_nodes == 0;
        has = true;
        acc.pb = pid;  // no hits yet
        last = 0xFFFFFFFFu;
        dvp[0] = dvp[1] = dvp[2] = (R)0;
        dpart = (R)0;
        if (!ray_meets_box<R>(ray, a.mesh)) {
          ++acc.particles;
          if (COUNT && a.rec.n_hits != nullptr) {
            a.rec.n_hits[pid] = 0;
            a.rec.truncated[pid] = 0;
#pragma unroll
            for (int i = 0; i < 3; ++i) a.rec.dv[3 * pid + i] = 0.0;
          }
          has = false;
        }
      }
      q_head = (q_head + take) & (kQueue - 1);
      q_count -= take;
      __syncwarp();
      if (take == 0) break;
    }

    // ---- 3. the warp is done when nothing is in flight and nothing is left to seed
    if (!__any_sync(kFull, has)) {
      if (drained && q_count == 0) break;
      continue;
    }

    // ---- 4. traversal round
    if constexpr (W > 2) {
      // Wide tree: lanes without triangles to test (searching) step through
      // nodes until each holds a triangle mask or has nothing left; lanes
      // that already hold one keep descending meanwhile (speculative), while
      // their stack has room for a postponed triangle group.  Then the
      // triangles.
      for (;;) {
        for (;;) {
          const bool work = has && !tdone;
          const bool search = work && tv.tm == 0u && ((tv.gx >> 24) != 0u || tv.sp > 0);
          if (!__any_sync(kFull, search)) break;
          if (search && (tv.gx >> 24) == 0u) travw_pop(tv, stack);
          const bool step = work && (tv.gx >> 24) != 0u &&
                            (tv.tm == 0u || tv.sp + (int)a.mesh.depth + 2 < kMaxStackW);
          if (step && (search || tv.tm != 0u)) travw_node<R, W>(a.mesh, ray, tv, stack, n_nodes, a.error);
        }
        if (has && !tdone) {
          if (tv.tm != 0u) travw_tris<R>(a.mesh, ray, last, tv, n_tris);
          tdone = (tv.gx >> 24) == 0u && tv.sp == 0;
        }
        const unsigned fin = __ballot_sync(kFull, has && tdone);
        const unsigned run = __ballot_sync(kFull, has && !tdone);
        if (run == 0u || (uint32_t)__popc(fin) >= a.refill_at) break;
      }
      continue;
    } else
    // ---- binary tree: inner nodes until every searching lane holds a leaf
    // (lanes with a leaf keep descending meanwhile), then the leaves
    for (;;) {
      // without staged nodes, the shared-memory check leaves the node loop
      if (n_stage == 0) {
        while (__any_sync(kFull, has && !tdone && tv.cur >= 0 && tv.leaf == 0)) {
          if (has && !tdone && tv.cur >= 0)
            trav_inner<R, false>(a.mesh, s_nodes, n_stage, ray, tv, stack, n_nodes, a.error);
        }
      } else {
        while (__any_sync(kFull, has && !tdone && tv.cur >= 0 && tv.leaf == 0)) {
          if (has && !tdone && tv.cur >= 0)
            trav_inner<R, true>(a.mesh, s_nodes, n_stage, ray, tv, stack, n_nodes, a.error);
        }
      }
      if (has && !tdone) {
        if (tv.leaf != 0) tdone = trav_leaf<R>(a.mesh, ray, last, tv, stack, n_tris);
        else if (tv.cur == kDone) tdone = true;
      }
      const unsigned fin = __ballot_sync(kFull, has && tdone);
      const unsigned run = __ballot_sync(kFull, has && !tdone);
      if (run == 0u || (uint32_t)__popc(fin) >= a.refill_at) break;
    }
  }
  if constexpr (COUNT) work_flush(a.acc, a.acc_stride, acc.q, n_nodes, n_tris, acc_stripe());
  warp_flush(a.acc, a.acc_stride, acc, acc_stripe());
}

// ---------------------------------------------------------- set-up kernel
__device__ double latitude_cdf_d(double x, double S, double K1, double D) {
  const double Sx = S * x;
  return (kSqrtPiD / (4.0 * S) * (2.0 * Sx * Sx + 1.0) * erfc(-Sx) + 0.5 * x * exp(-Sx * Sx) - K1) / D;
}
__device__ double latitude_pdf_d(double x, double S, double D) {
  const double Sx = S * x;
  return (exp(-Sx * Sx) + kSqrtPiD * Sx * erfc(-Sx)) / D;
}

// Block b prepares query b.  With `base` set, query b is a copy of *base whose
// direction / speed ratio come from dirs[b] / Svals[b] (when given) and whose
// Philox stream is base->stream_id + b; with `items` set, it also writes work
// item b = particles [0, N) of query b at work indices [b N, (b+1) N).
__global__ void setup_kernel(QueryDev* qs, const QueryDev* base, const double* dirs, const double* Svals,
                             ItemDev* items, const uint32_t* slots, AccStripe* acc, uint32_t acc_stride) {
  const uint32_t slot = slots != nullptr ? slots[blockIdx.x] : blockIdx.x;
  QueryDev& q = qs[slot];
  // the query's sums start at zero: its kAccStripes stripes of 16 words each
  for (uint32_t i = threadIdx.x; i < (uint32_t)kAccStripes * 16u; i += blockDim.x)
    reinterpret_cast<unsigned long long*>(&acc[(size_t)(i >> 4) * acc_stride + slot])[i & 15u] = 0ull;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int st = TPMC_OK;
    if (base != nullptr) {
      q = *base;
      q.stream_id = base->stream_id + blockIdx.x;
    }
    if (items != nullptr) {
      ItemDev it;
      it.g_begin = (uint64_t)blockIdx.x * q.N;
      it.pid_begin = 0;
      it.count = q.N;
      it.query = blockIdx.x;
      it.pad = 0;
      items[blockIdx.x] = it;
    }
    if (dirs != nullptr)
      for (int i = 0; i < 3; ++i) q.dir[i] = dirs[3 * blockIdx.x + i];
    const double c = sqrt(2.0 * kBoltz * q.T_inf / q.m);
    if (Svals != nullptr) q.V = Svals[blockIdx.x] * c;
    const double dn = sqrt(q.dir[0] * q.dir[0] + q.dir[1] * q.dir[1] + q.dir[2] * q.dir[2]);
    if (!(isfinite(q.V) && q.V > 0.0) || !(isfinite(dn) && dn > 0.0)) st = TPMC_EINVAL;
    const double S = q.V / c;
    if (!(S >= 0.01 && S <= 50.0)) st = TPMC_EINVAL;
    if (st == TPMC_OK) {
      q.S = S;
      q.c_mp = c;
      q.cw = sqrt(q.T_W / q.T_inf);
      double vh[3];
      for (int i = 0; i < 3; ++i) { vh[i] = q.dir[i] / dn; q.vhat[i] = vh[i]; }
      // Eq. 15: rotation about u = z x Vhat by beta = acos(z . Vhat), carrying +z onto Vhat.
      const double ux = -vh[1], uy = vh[0];  // z x Vhat = (-Vy, Vx, 0)
      const double sb = sqrt(ux * ux + uy * uy);
      const double cb = fmin(1.0, fmax(-1.0, vh[2]));
      double Rm[9];
      if (sb < 1e-12) {
        const double sg = cb > 0.0 ? 1.0 : -1.0;  // identity, or a half turn about x
        Rm[0] = 1; Rm[1] = 0; Rm[2] = 0; Rm[3] = 0; Rm[4] = sg; Rm[5] = 0; Rm[6] = 0; Rm[7] = 0; Rm[8] = sg;
      } else {
        const double kx = ux / sb, ky = uy / sb;  // unit axis (kx, ky, 0)
        const double beta = acos(cb);
        const double cs = cos(beta), sn = sin(beta), oc = 1.0 - cs;
        Rm[0] = cs + kx * kx * oc; Rm[1] = kx * ky * oc;      Rm[2] = ky * sn;
        Rm[3] = kx * ky * oc;      Rm[4] = cs + ky * ky * oc; Rm[5] = -kx * sn;
        Rm[6] = -ky * sn;          Rm[7] = kx * sn;           Rm[8] = cs;
      }
      for (int i = 0; i < 9; ++i) { q.R[i] = Rm[i]; q.fc[kFcR + i] = (float)Rm[i]; }
      const double eS = exp(-S * S), erS = erf(S);
      q.Dnorm = eS + kSqrtPiD * (1.0 + 2.0 * S * S) * erS / (2.0 * S);
      q.K1 = kSqrtPiD / (4.0 * S) * (2.0 * S * S + 1.0) * erfc(S) - 0.5 * eS;
      q.gamma = (kSqrtPiD * eS + (CUDART_PI / (2.0 * S) + CUDART_PI * S) * erS) * c * q.n * q.r_cv * q.r_cv;
      if (q.cv_kind != TPMC_CV_SPHERE) {
        // Rectangular CV (§I, §III.A): face f receives the flat-plate number
        // flux A_f n c G(s_f), G(s) = (e^{-s^2} + sqrt(pi) s erfc(-s)) / (2 sqrt(pi)),
        // and the particle ids up to floor(N C_{f+1}), C the cumulative share.
        double flux[6], total = 0.0;
        for (int f = 0; f < 6; ++f) {
          const int ax = f / 2, a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
          const double s_f = S * (f % 2 == 0 ? -vh[ax] : vh[ax]);
          const double area = (q.box_hi[a1] - q.box_lo[a1]) * (q.box_hi[a2] - q.box_lo[a2]);
          flux[f] = area * ((exp(-s_f * s_f) + kSqrtPiD * s_f * erfc(-s_f)) / (2.0 * kSqrtPiD));
          total += flux[f];
          q.face_s[f] = s_f;
          q.fface_s[f] = (float)s_f;
        }
        double cum = 0.0;
        for (int f = 0; f < 6; ++f) {
          cum += flux[f] / total;
          q.face_end[f] = f == 5 ? q.N : (uint64_t)floor((double)q.N * cum);
        }
        for (int i = 0; i < 3; ++i) {
          q.fbox_lo[i] = (float)q.box_lo[i];
          q.fbox_ext[i] = (float)(q.box_hi[i] - q.box_lo[i]);
        }
        q.gamma = total * c * q.n;
      }
      q.q_inf = 0.5 * q.n * q.m * q.V * q.V;
      // fixed point: worst case |v| <= max(S + 8, 8 c_W/c), so every int64 sum fits for
      // N * max_bounces hits of |dv| <= 2 |v|max and lever arms <= rmax.
      const double vmax = fmax(S + 8.0, 8.0 * q.cw);
      const double bound = (double)q.N * (double)q.max_bounces * 2.0 * 1.7320508075688772 * vmax * fmax(1.0, q.rmax);
      int shift = (int)floor(62.0 - log2(bound));
      shift = min(shift, 32);
      if (shift < 8) st = TPMC_EINVAL;
      q.shift = shift;
      q.quantum = ldexp(1.0, -shift);
      // squared drag contributions: a particle's |dv . Vhat| <= 2 vmax max_bounces,
      // so each quantised term stays below 2^62; the sum is a 128-bit integer
      const double dmax = 2.0 * vmax * (double)q.max_bounces;
      const int shift2 = max(0, min(32, (int)floor(62.0 - log2(dmax * dmax))));
      q.shift2 = shift2;
      q.quantum2 = ldexp(1.0, -shift2);
      q.fc[kFcScale2] = (float)ldexp(1.0, shift2);
      q.fc[kFcS] = (float)S;
      q.fc[kFcCw] = (float)q.cw;
      q.fc[kFcRcv] = (float)q.r_cv;
      q.fc[kFcSqrtpi4S] = (float)(kSqrtPiD / (4.0 * S));
      q.fc[kFcK1] = (float)q.K1;
      q.fc[kFcDinv] = (float)(1.0 / q.Dnorm);
      // tail-mass cubics of the latitude law at the poles (see latitude_pole):
      //   x -> +1: h(1) w - h'(1) w^2 / 2 + h''(1) w^3 / 6,  x -> -1: h(-1) w + h'(-1) w^2 / 2 + h''(-1) w^3 / 6,
      //   h(1) = [e^{-S^2} + sqrt(pi) S erfc(-S)] / D,  h(-1) = e^{-S^2} [1 - sqrt(pi) S erfcx(S)] / D,
      //   h'(+-1) = sqrt(pi) S erfc(-+S) / D,  h''(+-1) = 2 S^2 e^{-S^2} / D
      q.fc[kFcPole + 0] = (float)((eS + kSqrtPiD * S * erfc(-S)) / q.Dnorm);
      q.fc[kFcPole + 1] = (float)(-0.5 * kSqrtPiD * S * erfc(-S) / q.Dnorm);
      q.fc[kFcPole + 2] = (float)(S * S * eS / (3.0 * q.Dnorm));
      q.fc[kFcPole + 3] = (float)(eS * (1.0 - kSqrtPiD * S * erfcx(S)) / q.Dnorm);
      q.fc[kFcPole + 4] = (float)(0.5 * kSqrtPiD * S * erfc(S) / q.Dnorm);
      q.fc[kFcPole + 5] = (float)(S * S * eS / (3.0 * q.Dnorm));
      q.fc[kFcScale] = (float)ldexp(1.0, shift);
      for (int i = 0; i < 3; ++i) {
        q.fc[kFcVhat + i] = (float)vh[i];
        q.fc[kFcCenter + i] = (float)q.center[i];
        q.fc[kFcRef + i] = (float)q.ref[i];
      }
    }
    q.status = st;
    s_ok = st == TPMC_OK;
  }
  __syncthreads();
  if (!s_ok || q.cv_kind != TPMC_CV_SPHERE) return;  // the latitude table serves the sphere only
  const double S = q.S, K1 = q.K1, D = q.Dnorm;
  for (int j = threadIdx.x; j <= kHTable; j += blockDim.x) {
    double x;
    {
      const double zj = kZLo + (kZHi - kZLo) * j / kHTable;
      const double u = 0.5 * erfc(-zj * 0.70710678118654752440);  // Phi(z_j)
      double lo = -1.0, hi = 1.0;
      x = 2.0 * u - 1.0;
      for (int it = 0; it < 200; ++it) {
        const double f = latitude_cdf_d(x, S, K1, D) - u;
        if (f == 0.0) break;
        if (f < 0.0) lo = x; else hi = x;
        double xn = x - f / latitude_pdf_d(x, S, D);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        const double step = fabs(xn - x);
        x = xn;
        if (step < 1e-15) break;
      }
    }
    q.htab[j] = (float)x;
  }
}

// Normal-speed start table (FP64, once per context): entry (i, j) is the
// root of F(x; s_i) = Phi(z_j) by bisection, on the survival function above
// the median (the same law as Eq. 14a; see normal_speed_inverse).
__global__ void vn_table_kernel(float* tab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kVnNS * kVnNZ) return;
  const int i = k / kVnNZ, j = k % kVnNZ;
  const double s = kVnSLo + kVnStep * i;
  const double z = kZLo + kVnStep * j;
  const double u = 0.5 * erfc(-z * 0.70710678118654752440);
  const double sp = kSqrtPiD * s;
  const double Z = exp(-s * s) + sp * erfc(-s);
  double lo = 0.0, hi = fmax(s, 0.0) + 12.0;
  for (int it = 0; it < 200; ++it) {
    const double x = 0.5 * (lo + hi);
    if (x <= lo || x >= hi) break;
    const double y = x - s;
    bool below;
    if (u <= 0.5) {
      const double F = (exp(-s * s) - exp(-y * y) + sp * (erfc(-s) - erfc(y))) / Z;
      below = F < u;
    } else {
      const double Q = (exp(-y * y) + sp * erfc(y)) / Z;
      below = Q > 1.0 - u;
    }
    if (below) lo = x; else hi = x;
  }
  tab[k] = (float)(0.5 * (lo + hi));
}

// -------------------------------------------------------- final reduction
// Thread i reduces query slots[i] (or i) into out[i].
__global__ void finalize_kernel(const QueryDev* qs, const AccStripe* acc, uint32_t stride, uint32_t nq,
                                const uint32_t* slots, tpmc_result* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const uint32_t qi = slots != nullptr ? slots[i] : i;
  const QueryDev& q = qs[qi];
  // the stripes' sums; the squared-drag limbs as one exact 128-bit integer
  long long F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
  unsigned long long hits = 0, hitp = 0, trunc = 0, parts = 0, nodes = 0, tris = 0, d2lo = 0, d2hi = 0;
  for (int j = 0; j < kAccStripes; ++j) {
    const AccStripe& A = acc[(size_t)j * stride + qi];
    for (int k = 0; k < 3; ++k) { F[k] += A.F[k]; T[k] += A.T[k]; }
    hits += A.hits;
    hitp += A.hit_particles;
    trunc += A.truncated;
    parts += A.particles;
    nodes += A.nodes;
    tris += A.tris;
    const unsigned long long add_lo[3] = {A.d2[0], A.d2[1] << 30, A.d2[2] << 60};
    const unsigned long long add_hi[3] = {0ull, A.d2[1] >> 34, A.d2[2] >> 4};
    for (int k = 0; k < 3; ++k) {
      const unsigned long long nlo = d2lo + add_lo[k];
      d2hi += add_hi[k] + (nlo < d2lo ? 1ull : 0ull);
      d2lo = nlo;
    }
  }
  tpmc_result r;
  memset(&r, 0, sizeof(r));
  r.status = q.status;
  if (q.status == TPMC_OK) {
    const double Np = (double)parts;
    double sdv[3], srdv[3];
    for (int k = 0; k < 3; ++k) {
      sdv[k] = (double)F[k] * q.quantum;
      srdv[k] = (double)T[k] * q.quantum;
      r.sum_dv_q[k] = F[k];
      r.sum_rdv_q[k] = T[k];
    }
    // force = (Gamma/N) m c sum(dv) (§II.A); C_D = F . Vhat / (q_inf A_ref) (Eq. 1)
    const double scale = Np > 0 ? q.gamma / Np * q.m * q.c_mp : 0.0;
    for (int k = 0; k < 3; ++k) { r.force[k] = scale * sdv[k]; r.torque[k] = scale * srdv[k]; }
    r.CD = (r.force[0] * q.vhat[0] + r.force[1] * q.vhat[1] + r.force[2] * q.vhat[2]) / (q.q_inf * q.A_ref);
    // force and moment coefficient vectors (the moment about ref over q_inf A_ref l_ref, §III.D.1)
    for (int k = 0; k < 3; ++k) {
      r.CF[k] = r.force[k] / (q.q_inf * q.A_ref);
      r.CM[k] = r.torque[k] / (q.q_inf * q.A_ref * q.l_ref);
    }
    const double mean = Np > 0 ? (sdv[0] * q.vhat[0] + sdv[1] * q.vhat[1] + sdv[2] * q.vhat[2]) / Np : 0.0;
    const double d2 = ((double)d2hi * 18446744073709551616.0 + (double)d2lo) * q.quantum2;
    const double var = Np > 1 ? fmax(0.0, (d2 - Np * mean * mean) / (Np - 1.0)) : 0.0;
    r.CD_sigma = Np > 0 ? q.gamma * q.m * q.c_mp / (q.q_inf * q.A_ref) * sqrt(var / Np) : 0.0;
    r.S = q.S;
    r.S_W = q.S / q.cw;
    r.gamma = q.gamma;
    r.weight = Np > 0 ? q.gamma / Np : 0.0;
    r.q_inf = q.q_inf;
    r.c_mp = q.c_mp;
    r.r_cv = q.r_cv;
    for (int k = 0; k < 3; ++k) r.center[k] = q.center[k];
    r.fixed_quantum = q.quantum;
    r.n_particles = parts;
    r.n_hits = hits;
    r.n_hit_particles = hitp;
    r.n_truncated = trunc;
    r.n_node_visits = nodes;
    r.n_tri_tests = tris;
    if (parts != q.N) r.status = TPMC_ECUDA;
  }
  out[i] = r;
}

__global__ void panels_kernel(const QueryDev* q, const long long* panel, const double* frames64, uint32_t n_tri,
                              double* pressure, double* shear) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_tri) return;
  const double* f = frames64 + 8 * (size_t)i;
  const double area = f[3];
  double p = 0.0, s = 0.0;
  if (area > 0.0) {
    const double scale = q->gamma / (double)q->N * q->m * q->c_mp * q->quantum;
    double F[3];
    for (int k = 0; k < 3; ++k) F[k] = scale * (double)panel[3 * (size_t)i + k];
    const double fn = F[0] * f[0] + F[1] * f[1] + F[2] * f[2];
    p = -fn / area;
    const double tx = F[0] - fn * f[0], ty = F[1] - fn * f[1], tz = F[2] - fn * f[2];
    s = sqrt(tx * tx + ty * ty + tz * tz) / area;
  }
  if (pressure) pressure[i] = p;
  if (shear) shear[i] = s;
}

}  // namespace

// ------------------------------------------------------------- launchers
cudaError_t launch_setup(QueryDev* d_queries, uint32_t nq, const QueryDev* d_base, const double* d_dirs,
                         const double* d_S, ItemDev* d_items, const uint32_t* d_slots, AccStripe* d_acc,
                         uint32_t acc_stride, cudaStream_t stream) {
  if (nq == 0) return cudaSuccess;
  setup_kernel<<<nq, 160, 0, stream>>>(d_queries, d_base, d_dirs, d_S, d_items, d_slots, d_acc, acc_stride);
  return cudaGetLastError();
}

cudaError_t launch_vn_table(float* d_table, cudaStream_t stream) {
  vn_table_kernel<<<(kVnNS * kVnNZ + 127) / 128, 128, 0, stream>>>(d_table);
  return cudaGetLastError();
}

size_t trace_smem_bytes(const LaunchCfg& cfg, uint32_t n_nodes, uint32_t variant) {
  const uint32_t precision = variant & 1u;
  const size_t queue = (size_t)(cfg.block / 32) * kQueue *
                       (precision == TPMC_FP64 ? sizeof(Seeded<double>) : sizeof(Seeded<float>));
  const size_t staged =
      variant_width(variant) > 2 ? 0 : (size_t)std::min(cfg.smem_nodes, n_nodes) * kBinaryNodeF4 * sizeof(float4);
  return staged + queue + (size_t)cfg.block * sizeof(LaneAcc);
}

namespace {
using TraceFn = void (*)(TraceArgs);

// Kernel instantiation for a schedule: the register-capped float variants
// serve 128-thread blocks at 5 to 8 blocks per SM.
template <bool CLL, int W, bool COUNT>
TraceFn pick_trace_t(uint32_t precision, uint32_t block, uint32_t blocks_per_sm) {
  if (precision == TPMC_FP64) return trace_kernel<double, 0, CLL, W, COUNT>;
  if (block <= 128 && blocks_per_sm >= 8) return trace_kernel<float, 8, CLL, W, COUNT>;
  if (block <= 128 && blocks_per_sm == 7) return trace_kernel<float, 7, CLL, W, COUNT>;
  if (block <= 128 && blocks_per_sm == 6) return trace_kernel<float, 6, CLL, W, COUNT>;
  if (block <= 128 && blocks_per_sm == 5) return trace_kernel<float, 5, CLL, W, COUNT>;
  return trace_kernel<float, 0, CLL, W, COUNT>;
}

template <int W, bool COUNT>
TraceFn pick_trace_c(uint32_t variant, uint32_t block, uint32_t blocks_per_sm) {
  return (variant & kVariantCll) ? pick_trace_t<true, W, COUNT>(variant & 1u, block, blocks_per_sm)
                                 : pick_trace_t<false, W, COUNT>(variant & 1u, block, blocks_per_sm);
}

template <int W>
TraceFn pick_trace_w(uint32_t variant, uint32_t block, uint32_t blocks_per_sm) {
  return (variant & kVariantCount) ? pick_trace_c<W, true>(variant, block, blocks_per_sm)
                                   : pick_trace_c<W, false>(variant, block, blocks_per_sm);
}

TraceFn pick_trace(uint32_t variant, uint32_t block, uint32_t blocks_per_sm) {
  switch (variant_width(variant)) {
    case 8: return pick_trace_w<8>(variant, block, blocks_per_sm);
    case 4: return pick_trace_w<4>(variant, block, blocks_per_sm);
    default: return pick_trace_w<2>(variant, block, blocks_per_sm);
  }
}

int occupancy(TraceFn f, uint32_t block, size_t smem) {
  int nb = 0;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, (int)block, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}
}  // namespace

// Largest resident block count over the instantiations that can run `cfg`.
int trace_max_blocks_per_sm(uint32_t variant, const LaunchCfg& cfg, uint32_t n_nodes) {
  const size_t smem = trace_smem_bytes(cfg, n_nodes, variant);
  if (smem > 227 * 1024) return 0;
  int best = occupancy(pick_trace(variant, cfg.block, 1), cfg.block, smem);
  if ((variant & 1u) == TPMC_FP32 && cfg.block <= 128) {
    for (int minb : {5, 6, 7, 8}) {
      const int nb = occupancy(pick_trace(variant, cfg.block, (uint32_t)minb), cfg.block, smem);
      if (nb >= minb) best = std::max(best, nb);
    }
  }
  return best;
}

cudaError_t launch_trace(const TraceArgs& args, uint32_t variant, const LaunchCfg& cfg, int num_sms,
                         cudaStream_t stream) {
  // the mesh's own layout decides which traversal reads its nodes, and the
  // launch's counting flag whether the counters are compiled in
  variant = (variant & ~(kVariantWide4 | kVariantWide8 | kVariantCount)) |
            (args.mesh.width == 8 ? kVariantWide8 : (args.mesh.width == 4 ? kVariantWide4 : 0u)) |
            (args.count_work || args.rec.n_hits != nullptr || args.rec.tri != nullptr ? kVariantCount : 0u);
  const size_t smem = trace_smem_bytes(cfg, args.mesh.n_nodes, variant);
  const uint32_t grid = (uint32_t)num_sms * cfg.blocks_per_sm;
  const TraceFn f = pick_trace(variant, cfg.block, cfg.blocks_per_sm);
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  f<<<grid, cfg.block, smem, stream>>>(args);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const QueryDev* d_queries, const AccStripe* d_acc, uint32_t acc_stride, uint32_t nq,
                            const uint32_t* d_slots, tpmc_result* d_out, cudaStream_t stream) {
  if (nq == 0) return cudaSuccess;
  finalize_kernel<<<(nq + 127) / 128, 128, 0, stream>>>(d_queries, d_acc, acc_stride, nq, d_slots, d_out);
  return cudaGetLastError();
}

cudaError_t launch_panels(const QueryDev* d_query, const long long* d_panel, const float4*, const double* frames64,
                          uint32_t n_tri, double* d_pressure, double* d_shear, cudaStream_t stream) {
  if (n_tri == 0) return cudaSuccess;
  panels_kernel<<<(n_tri + 255) / 256, 256, 0, stream>>>(d_query, d_panel, frames64, n_tri, d_pressure, d_shear);
  return cudaGetLastError();
}

}  // namespace tpmc
