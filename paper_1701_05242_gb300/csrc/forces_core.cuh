// Per-particle force core shared by the single-system and batched force kernels.
#pragma once

#include <type_traits>

#include "dcm_internal.cuh"

namespace dcm {

constexpr int kForceBlock = 128;

template <typename R>
struct ForceArgs {
  Grid<R> g;
  R rc_max;
  int ntypes;
  R eps24[16], eps4[16], sig2[16];
  int shift;
};

__device__ __forceinline__ float recip(float x) {
  // hardware approximation refined by one Newton-Raphson step
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  float e = fmaf(-x, y, 1.0f);
  return fmaf(y, e, y);
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Loads of positions and cell starts in the pair walk.  NC: through the
// read-only (non-coherent) path, for kernels in which the arrays are never
// written; otherwise ordinary cached loads (ld.global.ca), for a kernel that
// wrote them earlier in the same launch behind a grid barrier.
template <bool NC>
__device__ __forceinline__ float4 ld_pos(const float4* p) {
  if constexpr (NC) return __ldg(p);
  else return __ldca(p);
}
template <bool NC>
__device__ __forceinline__ dvec4 ld_pos(const dvec4* p) {
  if constexpr (NC) {
    return ldg4(p);
  } else {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldca(q), b = __ldca(q + 1);
    return dvec4{a.x, a.y, b.x, b.y};
  }
}
template <bool NC>
__device__ __forceinline__ int32_t ld_start(const int32_t* p) {
  if constexpr (NC) return __ldg(p);
  else return __ldca(p);
}

// particle type stored as a number in w, clamped to [0, ntypes)
template <typename R>
__device__ __forceinline__ int type_of(R w, int ntypes) {
  int t = (int)w;
  return t < 0 ? 0 : (t >= ntypes ? ntypes - 1 : t);
}

// Half width of the sphere's x-window in a row.  Only the culling uses it,
// with a slack of 5e-4 cells on both ends, so in FP32 the one-instruction
// hardware square root suffices (its error is a few ulps).
__device__ __forceinline__ float window_half_width(float t) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
  return r;
}
__device__ __forceinline__ double window_half_width(double t) { return sqrt(t); }

// unwrapped cell index (no clamp) of a coordinate, used only for culling
template <typename R>
__device__ __forceinline__ int ufloor(R v) {
  return (int)floor(v);
}

// Accumulators of one particle.  One type: the constant factors are taken
// out of the pair loop: F = 24 sum s6 (2 s6 - 1) / r^2 r_ij, U = 4 sum
// (s6^2 - s6), r.F = 24 sum s6 (2 s6 - 1), with s6 = (1/r^2)^3.  Each pair's
// s6^2 - s6 is formed before summing: summing s6^2 and s6 separately and
// subtracting at the end loses the cancellation near r = sigma.  Several
// types: energy and virial per pair with the pair's eps and sigma.
template <typename R>
struct Acc {
  R fx = 0, fy = 0, fz = 0;
  R en = 0, vir = 0;
  int np = 0;
};

// Pairs of particle i (coordinates xi, yi, zi in the image frame of the
// segment) with sorted particles [lo, hi).  SJ: the segment's j coordinates
// need the exact -L image shift (sh); otherwise they are used as loaded.
template <typename R, bool SJ, bool TYPED, bool NC = true>
__device__ __forceinline__ void pair_range(const typename RT<R>::R4* __restrict__ pos, int lo, int hi, R xi, R yi,
                                           R zi, R shx, R shy, R shz, R rc2, int ti, const ForceArgs<R>& a,
                                           const R* ushift, Acc<R>& c) {
#pragma unroll 2
  for (int j = lo; j < hi; ++j) {
    auto pj = ld_pos<NC>(pos + j);
    R dx, dy, dz;
    if (SJ) {
      dx = xi - (pj.x + shx);
      dy = yi - (pj.y + shy);
      dz = zi - (pj.z + shz);
    } else {
      dx = xi - pj.x;
      dy = yi - pj.y;
      dz = zi - pj.z;
    }
    R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    bool acc = r2 < rc2;
    R inv = recip(r2);
    inv = acc ? inv : (R)0;
    if (TYPED) {
      int tj = type_of(pj.w, a.ntypes);
      int tp = ti * a.ntypes + tj;
      R s2 = a.sig2[tp] * inv;
      R s6 = s2 * s2 * s2;
      R pv = a.eps24[tp] * s6 * fma((R)2, s6, (R)-1);  // r . F_ij
      R fs = pv * inv;
      c.fx = fma(fs, dx, c.fx);
      c.fy = fma(fs, dy, c.fy);
      c.fz = fma(fs, dz, c.fz);
      R us = tj == 0 ? ushift[0] : (tj == 1 ? ushift[1] : (tj == 2 ? ushift[2] : ushift[3]));
      R u = a.eps4[tp] * s6 * (s6 - (R)1);
      c.en += acc ? u - us : (R)0;
      c.vir += pv;
    } else {
      R s6 = inv * inv * inv;
      R pv = s6 * fma((R)2, s6, (R)-1);  // r . F_ij / 24
      R q = pv * inv;                    // |F_ij| / (24 r)
      c.fx = fma(q, dx, c.fx);
      c.fy = fma(q, dy, c.fy);
      c.fz = fma(q, dz, c.fz);
      c.en += fma(s6, s6, -s6);          // U / 4
      c.vir += pv;
    }
    c.np += acc ? 1 : 0;
  }
}

// Packed form of the one-type FP32 pair loop: candidates j and j + 1 of a
// segment share every arithmetic instruction that has an FP32x2 form (FMA,
// MUL, ADD); the comparison, the hardware reciprocal and the select stay
// scalar.  An odd segment's last pair slot repeats its last candidate and is
// masked out.  Signs: with d = r_j - r_i (no packed operand needs negating),
// y = 1/r^2 (zero when rejected) and s6 = y^3,
//   r.F/24 = s6 (2 s6 - 1),   -F_i/24 = sum (r.F/24) y d,   U/4 = s6 (s6 - 1),
// and the reciprocal is refined exactly as recip() does.
struct Acc2 {
  float2 fx = {0.f, 0.f}, fy = {0.f, 0.f}, fz = {0.f, 0.f};
  float2 en = {0.f, 0.f}, vir = {0.f, 0.f};
  int np = 0;
};

// Per-particle accumulation forms of the mixed precision form (the values
// of dcm_params.accumulation).  The pair loops always sum into short-lived
// partials (Acc for the scalar loop, Acc2 for the packed one); the long-lived
// sums S of the form take them over:
//   kPlain      no S: the partials are the sums (plain FP32);
//   kRowF64     after every row segment the partials are added into FP64 sums;
//   kRowKahan   ... into FP32 sums with Kahan compensation;
//   kPlaneF64, kPlaneKahan  the same once per z-plane of the stencil (the
//               partials then span the plane's rows: up to five at rc = 3);
//   kPairKahan  every pair term goes into the partials with Kahan compensation
//               (S holds the compensation of each packed lane);
//   kPairF64    every pair term is added into FP64 sums (the partials stay 0).
enum class Accum : int {
  kPlain = DCM_ACC_FP32,
  kRowF64 = DCM_ACC_ROW_FP64,
  kRowKahan = DCM_ACC_ROW_KAHAN,
  kPairKahan = DCM_ACC_PAIR_KAHAN,
  kPairF64 = DCM_ACC_PAIR_FP64,
  kPlaneF64 = DCM_ACC_PLANE_FP64,
  kPlaneKahan = DCM_ACC_PLANE_KAHAN
};
constexpr bool row_form(Accum m) { return m == Accum::kRowF64 || m == Accum::kRowKahan; }
constexpr bool plane_form(Accum m) { return m == Accum::kPlaneF64 || m == Accum::kPlaneKahan; }
// forms whose pair loop is the plain one (the partials are taken over later or never)
constexpr bool plain_loop(Accum m) { return m == Accum::kPlain || row_form(m) || plane_form(m); }
constexpr bool f64_form(Accum m) { return m == Accum::kRowF64 || m == Accum::kPairF64 || m == Accum::kPlaneF64; }

template <Accum M>
using AccumTag = std::integral_constant<Accum, M>;

// Call f(AccumTag<M>{}) for the form acc (a DCM_ACC_* value, AUTO resolved).
// The scalar loop (X2 false) runs no pair form: its callers resolve those to
// the row forms first.
template <bool X2, typename F>
__host__ auto with_accum(int acc, F&& f) {
  switch (acc) {
    case DCM_ACC_FP32: return f(AccumTag<Accum::kPlain>{});
    case DCM_ACC_ROW_FP64: return f(AccumTag<Accum::kRowF64>{});
    case DCM_ACC_ROW_KAHAN: return f(AccumTag<Accum::kRowKahan>{});
    case DCM_ACC_PLANE_FP64: return f(AccumTag<Accum::kPlaneF64>{});
    case DCM_ACC_PAIR_KAHAN:
      if constexpr (X2) return f(AccumTag<Accum::kPairKahan>{});
      else return f(AccumTag<Accum::kRowKahan>{});
    case DCM_ACC_PAIR_FP64:
      if constexpr (X2) return f(AccumTag<Accum::kPairF64>{});
      else return f(AccumTag<Accum::kRowF64>{});
    default: return f(AccumTag<Accum::kPlaneKahan>{});
  }
}

// The five sums of a particle, in this order: fx, fy, fz, en, vir.
template <Accum M>
struct Sums {};
template <>
struct Sums<Accum::kRowF64> {
  double v[5] = {0, 0, 0, 0, 0};
};
template <>
struct Sums<Accum::kPairF64> {
  double v[5] = {0, 0, 0, 0, 0};
};
template <>
struct Sums<Accum::kPlaneF64> {
  double v[5] = {0, 0, 0, 0, 0};
};
template <>
struct Sums<Accum::kRowKahan> {
  float s[5] = {0, 0, 0, 0, 0}, k[5] = {0, 0, 0, 0, 0};
};
template <>
struct Sums<Accum::kPlaneKahan> {
  float s[5] = {0, 0, 0, 0, 0}, k[5] = {0, 0, 0, 0, 0};
};
template <>
struct Sums<Accum::kPairKahan> {
  float2 k[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
};

// Kahan's compensated summation (Kahan 1965): s accumulates, k carries the
// rounding error of the last addition (the amount s holds too much), so the
// compensated value of the sum is s - k.  Neither form is reassociated by the
// compiler (no fast-math).
__device__ __forceinline__ void kahan_add(float& s, float& k, float x) {
  const float y = x - k;
  const float u = s + y;
  k = (u - s) - y;
  s = u;
}
__device__ __forceinline__ void kahan_add2(float2& s, float2& k, float2 x) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 y = __ffma2_rn(k, m1, x);  // x - k, exact negation
  const float2 u = __fadd2_rn(s, y);
  k = __ffma2_rn(y, m1, __ffma2_rn(s, m1, u));  // (u - s) - y
  s = u;
}

// Fold the partials into the sums of a row or plane form and clear them
// (without EW only the force components: energy and virial are not summed).
template <Accum M, typename R, bool X2, bool EW = true>
__device__ __forceinline__ void flush_partials(Acc<R>& c, Acc2& c2, Sums<M>& S) {
  if constexpr (row_form(M) || plane_form(M)) {
    float v[5];
    if constexpr (X2) {
      v[0] = c2.fx.x + c2.fx.y;
      v[1] = c2.fy.x + c2.fy.y;
      v[2] = c2.fz.x + c2.fz.y;
      v[3] = c2.en.x + c2.en.y;
      v[4] = c2.vir.x + c2.vir.y;
      c2.fx = c2.fy = c2.fz = c2.en = c2.vir = make_float2(0.f, 0.f);
    } else {
      v[0] = c.fx;
      v[1] = c.fy;
      v[2] = c.fz;
      v[3] = c.en;
      v[4] = c.vir;
      c.fx = c.fy = c.fz = c.en = c.vir = (R)0;
    }
#pragma unroll
    for (int q = 0; q < (EW ? 5 : 3); ++q) {
      if constexpr (f64_form(M))
        S.v[q] += (double)v[q];
      else
        kahan_add(S.s[q], S.k[q], v[q]);
    }
  }
}


// Add the packed terms of one step (force components, U/4 or U, r.F) into
// the partials or the sums of form M.
template <Accum M, bool EW = true>
__device__ __forceinline__ void add_terms2(Acc2& c, Sums<M>& S, float2 q, float2 dx, float2 dy, float2 dz,
                                           float2 en, float2 pv) {
  if constexpr (M == Accum::kPairKahan) {
    kahan_add2(c.fx, S.k[0], __fmul2_rn(q, dx));
    kahan_add2(c.fy, S.k[1], __fmul2_rn(q, dy));
    kahan_add2(c.fz, S.k[2], __fmul2_rn(q, dz));
    if constexpr (EW) {
      kahan_add2(c.en, S.k[3], en);
      kahan_add2(c.vir, S.k[4], pv);
    }
  } else if constexpr (M == Accum::kPairF64) {
    const float2 t0 = __fmul2_rn(q, dx), t1 = __fmul2_rn(q, dy), t2 = __fmul2_rn(q, dz);
    S.v[0] += (double)t0.x + (double)t0.y;
    S.v[1] += (double)t1.x + (double)t1.y;
    S.v[2] += (double)t2.x + (double)t2.y;
    if constexpr (EW) {
      S.v[3] += (double)en.x + (double)en.y;
      S.v[4] += (double)pv.x + (double)pv.y;
    }
  } else {
    c.fx = __ffma2_rn(q, dx, c.fx);
    c.fy = __ffma2_rn(q, dy, c.fy);
    c.fz = __ffma2_rn(q, dz, c.fz);
    if constexpr (EW) {
      c.en = __fadd2_rn(c.en, en);
      c.vir = __fadd2_rn(c.vir, pv);
    }
  }
}

// One packed step on the differences d = r_j - r_i of two candidates (m0,
// m1: whether each slot holds a real candidate).  Without EW the step sums
// the force only (no energy, virial or pair count).
template <Accum M, bool EW = true>
__device__ __forceinline__ void pair_x2_d(float2 dx, float2 dy, float2 dz, bool m0, bool m1, float rc2, Acc2& c,
                                          Sums<M>& S) {
  const float2 two = make_float2(2.f, 2.f), m1f = make_float2(-1.f, -1.f);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  float y0, y1;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(r2.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(r2.y));
  float2 y = make_float2(y0, y1);
  const float2 e = __ffma2_rn(make_float2(-r2.x, -r2.y), y, make_float2(1.f, 1.f));
  y = __ffma2_rn(y, e, y);
  const bool a0 = m0 && r2.x < rc2, a1 = m1 && r2.y < rc2;
  y = make_float2(a0 ? y.x : 0.f, a1 ? y.y : 0.f);
  const float2 s6 = __fmul2_rn(__fmul2_rn(y, y), y);
  const float2 pv = __fmul2_rn(s6, __ffma2_rn(s6, two, m1f));  // r.F / 24
  const float2 q = __fmul2_rn(pv, y);
  if constexpr (plain_loop(M)) {
    // the plain step, fused: c.en += s6 (s6 - 1)
    c.fx = __ffma2_rn(q, dx, c.fx);
    c.fy = __ffma2_rn(q, dy, c.fy);
    c.fz = __ffma2_rn(q, dz, c.fz);
    if constexpr (EW) {
      c.en = __ffma2_rn(s6, __fadd2_rn(s6, m1f), c.en);
      c.vir = __fadd2_rn(c.vir, pv);
    }
  } else {
    add_terms2<M, EW>(c, S, q, dx, dy, dz, EW ? __fmul2_rn(s6, __fadd2_rn(s6, m1f)) : s6, pv);
  }
  if constexpr (EW) c.np += (int)a0 + (int)a1;
}

// One packed step: candidates p0 and p1 against particle i.
template <bool SJ, Accum M, bool EW = true>
__device__ __forceinline__ void pair_x2(const float4& p0, const float4& p1, bool m0, bool m1, float xi, float yi,
                                        float zi, float shx, float shy, float shz, float rc2, Acc2& c,
                                        Sums<M>& S) {
  float2 dx, dy, dz;
  if (SJ) {
    dx = make_float2((p0.x + shx) - xi, (p1.x + shx) - xi);
    dy = make_float2((p0.y + shy) - yi, (p1.y + shy) - yi);
    dz = make_float2((p0.z + shz) - zi, (p1.z + shz) - zi);
  } else {
    dx = make_float2(p0.x - xi, p1.x - xi);
    dy = make_float2(p0.y - yi, p1.y - yi);
    dz = make_float2(p0.z - zi, p1.z - zi);
  }
  pair_x2_d<M, EW>(dx, dy, dz, m0, m1, rc2, c, S);
}

// The packed step for up to two types: the constants of the pair type of
// each slot (sigma^2, 24 eps, 4 eps and the energy shift) are picked from the
// two of particle i's row by the slot's type; m0, m1 as in pair_x2_d.
template <Accum M, bool EW = true>
__device__ __forceinline__ void pair_x2_dt(float2 dx, float2 dy, float2 dz, bool m0, bool m1, float rc2, float2 sg,
                                           float2 e24, float2 e4, float2 us, Acc2& c, Sums<M>& S) {
  const float2 two = make_float2(2.f, 2.f), m1f = make_float2(-1.f, -1.f);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  float y0, y1;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(r2.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(r2.y));
  float2 y = make_float2(y0, y1);
  const float2 e = __ffma2_rn(make_float2(-r2.x, -r2.y), y, make_float2(1.f, 1.f));
  y = __ffma2_rn(y, e, y);
  const bool a0 = m0 && r2.x < rc2, a1 = m1 && r2.y < rc2;
  y = make_float2(a0 ? y.x : 0.f, a1 ? y.y : 0.f);
  us = make_float2(a0 ? us.x : 0.f, a1 ? us.y : 0.f);
  const float2 s2 = __fmul2_rn(sg, y);
  const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2);
  const float2 pv = __fmul2_rn(e24, __fmul2_rn(s6, __ffma2_rn(s6, two, m1f)));  // r . F_ij
  const float2 q = __fmul2_rn(pv, y);
  const float2 u =
      EW ? __ffma2_rn(e4, __fmul2_rn(s6, __fadd2_rn(s6, m1f)), make_float2(-us.x, -us.y)) : make_float2(0.f, 0.f);
  if constexpr (plain_loop(M)) {
    c.fx = __ffma2_rn(q, dx, c.fx);
    c.fy = __ffma2_rn(q, dy, c.fy);
    c.fz = __ffma2_rn(q, dz, c.fz);
    if constexpr (EW) {
      c.en = __fadd2_rn(c.en, u);
      c.vir = __fadd2_rn(c.vir, pv);
    }
  } else {
    add_terms2<M, EW>(c, S, q, dx, dy, dz, u, pv);
  }
  if constexpr (EW) c.np += (int)a0 + (int)a1;
}

// Typed form of pair_range_x2 for one or two types.  k8 holds particle i's
// row: k8[t] the energy shift, k8[2 + t] sigma^2, k8[4 + t] 24 eps, k8[6 + t]
// 4 eps of the pair type (type of i, t); a candidate's type is 1 if its w is
// at least 1 (type_of clamped to two types), and with one type both columns
// are equal.
template <bool SJ, Accum M, bool NC = true, bool EW = true>
__device__ __forceinline__ void pair_range_x2t(const float4* __restrict__ pos, int lo, int hi, float xi, float yi,
                                               float zi, float shx, float shy, float shz, float rc2,
                                               const float* k8, Acc2& c, Sums<M>& S) {
  for (int j = lo; j < hi; j += 2) {
    const bool has1 = j + 1 < hi;
    const int j1 = has1 ? j + 1 : j;
    const float4 p0 = ld_pos<NC>(pos + j), p1 = ld_pos<NC>(pos + j1);
    float2 dx, dy, dz;
    if (SJ) {
      dx = make_float2((p0.x + shx) - xi, (p1.x + shx) - xi);
      dy = make_float2((p0.y + shy) - yi, (p1.y + shy) - yi);
      dz = make_float2((p0.z + shz) - zi, (p1.z + shz) - zi);
    } else {
      dx = make_float2(p0.x - xi, p1.x - xi);
      dy = make_float2(p0.y - yi, p1.y - yi);
      dz = make_float2(p0.z - zi, p1.z - zi);
    }
    const bool t0 = p0.w >= 1.f, t1 = p1.w >= 1.f;
    pair_x2_dt<M, EW>(dx, dy, dz, true, has1, rc2, make_float2(t0 ? k8[3] : k8[2], t1 ? k8[3] : k8[2]),
               make_float2(t0 ? k8[5] : k8[4], t1 ? k8[5] : k8[4]), make_float2(t0 ? k8[7] : k8[6], t1 ? k8[7] : k8[6]),
               make_float2(t0 ? k8[1] : k8[0], t1 ? k8[1] : k8[0]), c, S);
  }
}

template <bool SJ, Accum M, bool NC = true, bool EW = true>
__device__ __forceinline__ void pair_range_x2(const float4* __restrict__ pos, int lo, int hi, float xi, float yi,
                                              float zi, float shx, float shy, float shz, float rc2, Acc2& c,
                                              Sums<M>& S) {
  for (int j = lo; j < hi; j += 2) {
    const bool has1 = j + 1 < hi;
    const int j1 = has1 ? j + 1 : j;
    const float4 p0 = ld_pos<NC>(pos + j), p1 = ld_pos<NC>(pos + j1);
    pair_x2<SJ, M, EW>(p0, p1, true, has1, xi, yi, zi, shx, shy, shz, rc2, c, S);
  }
}

// Segment dispatch: the packed loop for FP32 (one type, or up to two types
// with the row constants in ushift[0 .. 7]), the scalar loop otherwise; the
// row forms of accumulation take the segment's partials over at its end.
template <typename R, bool SJ, bool TYPED, bool X2, Accum M, bool NC = true, bool EW = true>
__device__ __forceinline__ void segment(const typename RT<R>::R4* __restrict__ pos, int lo, int hi, R xi, R yi, R zi,
                                        R shx, R shy, R shz, R rc2, int ti, const ForceArgs<R>& a, const R* ushift,
                                        Acc<R>& c, Acc2& c2, Sums<M>& S) {
  if constexpr (X2 && TYPED) {
    pair_range_x2t<SJ, M, NC, EW>(pos, lo, hi, xi, yi, zi, shx, shy, shz, rc2, ushift, c2, S);
  } else if constexpr (X2) {
    pair_range_x2<SJ, M, NC, EW>(pos, lo, hi, xi, yi, zi, shx, shy, shz, rc2, c2, S);
  } else {
    pair_range<R, SJ, TYPED, NC>(pos, lo, hi, xi, yi, zi, shx, shy, shz, rc2, ti, a, ushift, c);
  }
  if constexpr (row_form(M)) flush_partials<M, R, X2, EW>(c, c2, S);
}

// Which segments of the row walk are evaluated: all of them, or only those
// that reach a periodic image (a row outside the grid in y or z, or the part
// of a window beyond either x end).
enum class Walk { kAll, kImagesOnly };

// The culled cell-row walk of particle `self` (position pi, clamped cutoff
// rci) over the cell grid g whose cell starts are start[0 .. ncell] (positions
// pos sorted by cell), accumulating into c (scalar loop) or c2 (packed).
template <typename R, bool TYPED, bool X2, Accum M, bool NC = true, Walk MODE = Walk::kAll, bool EW = true>
__device__ __forceinline__ void walk_rows(const typename RT<R>::R4* __restrict__ pos,
                                          const int32_t* __restrict__ start, const Grid<R>& g,
                                          const ForceArgs<R>& a, int self, const typename RT<R>::R4& pi, R rci,
                                          int ti, const R* ushift, Acc<R>& c, Acc2& c2, Sums<M>& S) {
  constexpr bool kImg = MODE == Walk::kImagesOnly;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const R l = g.edge, il = g.inv_edge, ilx = g.inv_edge_x;
  const R rc2 = rci * rci;
  const R rc2s = rc2 * (R)1.000004;  // culling slack; the pair test is exact
  const int cx = cell_coord<R>(pi.x, g.edge_x, ilx, nx);
  const int cy = cell_coord<R>(pi.y, l, il, ny);
  const int cz = cell_coord<R>(pi.z, l, il, nz);
  const int H = (int)ceil(rci * il), Hx = (int)ceil(rci * ilx);
  for (int uz = cz - H; uz <= cz + H; ++uz) {
    R gz = uz > cz ? (R)uz * l - pi.z : (uz < cz ? pi.z - (R)(uz + 1) * l : (R)0);
    R gz2 = gz * gz;
    if (gz2 >= rc2s) continue;
    int wz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
    R zi = uz >= nz ? pi.z - g.L[2] : pi.z;  // image +L: shift i
    R zsh = uz < 0 ? -g.L[2] : (R)0;          // image -L: shift j
    for (int uy = cy - H; uy <= cy + H; ++uy) {
      R gy = uy > cy ? (R)uy * l - pi.y : (uy < cy ? pi.y - (R)(uy + 1) * l : (R)0);
      R gyz2 = gz2 + gy * gy;
      if (gyz2 >= rc2s) continue;
      int wy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
      R yi = uy >= ny ? pi.y - g.L[1] : pi.y;
      R ysh = uy < 0 ? -g.L[1] : (R)0;
      R wx = window_half_width(rc2s - gyz2);
      int ulo = ufloor<R>((pi.x - wx) * ilx - (R)5e-4);
      int uhi = ufloor<R>((pi.x + wx) * ilx + (R)5e-4);
      // both ends clamped into [cx - Hx - 1, cx + Hx + 1]: for a coordinate
      // outside [0, L) (its cell clamped into the grid, its window not) the
      // segments come out empty and every index stays in range
      ulo = min(max(ulo, cx - Hx), cx + Hx + 1);
      uhi = max(min(uhi, cx + Hx), cx - Hx - 1);
      // 32-bit: parameter validation keeps the cell count below 2^31 - 1
      const int row = nx * (wy + ny * wz);
      // segment u < 0: image -L (shift j)
      if (ulo < 0) {
        int a1 = min(uhi, -1);
        int j0 = ld_start<NC>(start + row + ulo + nx), j1 = ld_start<NC>(start + row + a1 + nx + 1);
        segment<R, true, TYPED, X2, M, NC, EW>(pos, j0, j1, pi.x, yi, zi, -g.L[0], ysh, zsh, rc2, ti, a, ushift, c, c2, S);
      }
      // segment 0 <= u < nx: no x shift; the particle itself is skipped
      const bool img_row = uy < 0 || uy >= ny || uz < 0 || uz >= nz;
      if (!kImg || img_row) {
        int a0 = max(ulo, 0), a1 = min(uhi, nx - 1);
        if (a0 <= a1) {
          int j0 = ld_start<NC>(start + row + a0), j1 = ld_start<NC>(start + row + a1 + 1);
          if (!kImg && uy == cy && uz == cz) {  // the particle's own row: cut it out
            segment<R, false, TYPED, X2, M, NC, EW>(pos, j0, min(j1, self), pi.x, yi, zi, 0, 0, 0, rc2, ti, a, ushift, c, c2, S);
            segment<R, false, TYPED, X2, M, NC, EW>(pos, max(j0, self + 1), j1, pi.x, yi, zi, 0, 0, 0, rc2, ti, a, ushift, c,
                                         c2, S);
          } else if (ysh == (R)0 && zsh == (R)0) {
            segment<R, false, TYPED, X2, M, NC, EW>(pos, j0, j1, pi.x, yi, zi, 0, 0, 0, rc2, ti, a, ushift, c, c2, S);
          } else {
            segment<R, true, TYPED, X2, M, NC, EW>(pos, j0, j1, pi.x, yi, zi, (R)0, ysh, zsh, rc2, ti, a, ushift, c, c2, S);
          }
        }
      }
      // segment u >= nx: image +L (shift i)
      if (uhi >= nx) {
        int a0 = max(ulo, nx);
        int j0 = ld_start<NC>(start + row + a0 - nx), j1 = ld_start<NC>(start + row + uhi - nx + 1);
        segment<R, true, TYPED, X2, M, NC, EW>(pos, j0, j1, pi.x - g.L[0], yi, zi, (R)0, ysh, zsh, rc2, ti, a, ushift, c, c2, S);
      }
    }
    if constexpr (plane_form(M)) flush_partials<M, R, X2, EW>(c, c2, S);
  }
}

// Cutoffs outside [0, rc_max] (or NaN) are clamped: the stencil then never
// reaches past one periodic image, which keeps every cell index in range.
template <typename R>
__device__ __forceinline__ R clamp_cutoff(R rc_in, R rc_max) {
  R rci = rc_in;
  if (!(rci <= rc_max)) rci = rc_max;
  if (!(rci > (R)0)) rci = (R)0;
  return rci;
}

// Forces, energy and virial of particle `self` (position pi, cutoff rc_in)
// over the cell grid g whose cell starts are start[0 .. ncell] (positions
// pos, sorted by cell), with the per-particle sums of accumulation form M.
// Returns the force and writes e_i, w_i (in FP64: the totals are reduced
// from them in FP64) and the accepted-pair count.
// Without EW (the packed loop only) the energy, the virial and the pair
// count are not summed: e_out, w_out, np_out and the force's w are zero.
template <typename R, bool TYPED, bool X2 = false, Accum M = Accum::kPlain, bool NC = true, bool EW = true>
__device__ __forceinline__ typename RT<R>::R4 force_one(const typename RT<R>::R4* __restrict__ pos,
                                                        const int32_t* __restrict__ start, const Grid<R>& g,
                                                        const ForceArgs<R>& a, int self,
                                                        const typename RT<R>::R4& pi, R rc_in, double& e_out,
                                                        double& w_out, int& np_out) {
  static_assert(!X2 || sizeof(R) == 4, "the packed loop serves FP32 only (with types: at most two)");
  static_assert(M == Accum::kPlain || sizeof(R) == 4, "accumulation forms apply to FP32 pair math only");
  static_assert(X2 || plain_loop(M), "the pair forms run on the packed loop");
  Acc<R> c;
  Acc2 c2;
  Sums<M> S;
  const R rci = clamp_cutoff<R>(rc_in, a.rc_max);
  const R rc2 = rci * rci;
  const int ti = TYPED ? type_of(pi.w, a.ntypes) : 0;
  R ushift[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (a.shift && rc2 > (R)0) {  // no pairs at rc = 0: no shift either
    for (int t = 0; t < (TYPED ? a.ntypes : 1); ++t) {
      int tp = ti * a.ntypes + t;
      R s2 = (TYPED ? a.sig2[tp] : (R)1) / rc2;
      R s6 = s2 * s2 * s2;
      ushift[t] = (TYPED ? a.eps4[tp] : (R)4) * s6 * (s6 - (R)1);
    }
  }
  if constexpr (X2 && TYPED) {  // particle i's row for the packed typed loop (one or two types)
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int tc = t < a.ntypes ? t : a.ntypes - 1, tp = ti * a.ntypes + tc;
      ushift[t] = ushift[tc];
      ushift[2 + t] = a.sig2[tp];
      ushift[4 + t] = a.eps24[tp];
      ushift[6 + t] = a.eps4[tp];
    }
  }
  static_assert(EW || X2, "the scalar loop always sums energy and virial");
  walk_rows<R, TYPED, X2, M, NC, Walk::kAll, EW>(pos, start, g, a, self, pi, rci, ti, ushift, c, c2, S);
  // The five sums (fx, fy, fz, en, vir) of the form, in FP64 where the form
  // keeps them so; the packed loop sums the sign-flipped differences r_j - r_i.
  using V = std::conditional_t<f64_form(M), double, R>;
  V v[5];
  const int np = X2 ? c2.np : c.np;
  if constexpr (f64_form(M)) {
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] = S.v[q];
  } else if constexpr (M == Accum::kRowKahan || M == Accum::kPlaneKahan) {
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] = S.s[q] - S.k[q];
  } else if constexpr (M == Accum::kPairKahan) {
    const float2 p[5] = {c2.fx, c2.fy, c2.fz, c2.en, c2.vir};
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] = (p[q].x - S.k[q].x) + (p[q].y - S.k[q].y);
  } else if constexpr (X2) {  // plain: fold the two packed lanes
    v[0] = c2.fx.x + c2.fx.y;
    v[1] = c2.fy.x + c2.fy.y;
    v[2] = c2.fz.x + c2.fz.y;
    v[3] = c2.en.x + c2.en.y;
    v[4] = c2.vir.x + c2.vir.y;
  } else {
    v[0] = c.fx;
    v[1] = c.fy;
    v[2] = c.fz;
    v[3] = c.en;
    v[4] = c.vir;
  }
  const V sgn = X2 ? (V)-1 : (V)1;
  typename RT<R>::R4 out;
  if (TYPED) {
    out.x = (R)(sgn * v[0]);
    out.y = (R)(sgn * v[1]);
    out.z = (R)(sgn * v[2]);
    e_out = (double)((V)0.5 * v[3]);
    w_out = (double)((V)0.5 * v[4]);
  } else {
    out.x = (R)((V)24 * sgn * v[0]);
    out.y = (R)((V)24 * sgn * v[1]);
    out.z = (R)((V)24 * sgn * v[2]);
    e_out = (double)((V)2 * v[3] - (V)0.5 * (V)np * (V)ushift[0]);
    w_out = (double)((V)12 * v[4]);
  }
  if constexpr (!EW) {
    e_out = w_out = 0.0;
    np_out = 0;
    out.w = (R)0;
    return out;
  }
  out.w = (R)e_out;
  np_out = np;
  return out;
}

}  // namespace dcm
