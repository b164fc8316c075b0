// Per-particle force core shared by the single-system and batched force kernels.
#pragma once

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
template <typename R, bool SJ, bool TYPED>
__device__ __forceinline__ void pair_range(const typename RT<R>::R4* __restrict__ pos, int lo, int hi, R xi, R yi,
                                           R zi, R shx, R shy, R shz, R rc2, int ti, const ForceArgs<R>& a,
                                           const R* ushift, Acc<R>& c) {
#pragma unroll 2
  for (int j = lo; j < hi; ++j) {
    auto pj = ldg4(pos + j);
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

// One packed step on the differences d = r_j - r_i of two candidates (m0,
// m1: whether each slot holds a real candidate).
__device__ __forceinline__ void pair_x2_d(float2 dx, float2 dy, float2 dz, bool m0, bool m1, float rc2, Acc2& c) {
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
  c.fx = __ffma2_rn(q, dx, c.fx);
  c.fy = __ffma2_rn(q, dy, c.fy);
  c.fz = __ffma2_rn(q, dz, c.fz);
  c.en = __ffma2_rn(s6, __fadd2_rn(s6, m1f), c.en);
  c.vir = __fadd2_rn(c.vir, pv);
  c.np += (int)a0 + (int)a1;
}

// One packed step: candidates p0 and p1 against particle i.
template <bool SJ>
__device__ __forceinline__ void pair_x2(const float4& p0, const float4& p1, bool m0, bool m1, float xi, float yi,
                                        float zi, float shx, float shy, float shz, float rc2, Acc2& c) {
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
  pair_x2_d(dx, dy, dz, m0, m1, rc2, c);
}

// The packed step for up to two types: the constants of the pair type of
// each slot (sigma^2, 24 eps, 4 eps and the energy shift) are picked from the
// two of particle i's row by the slot's type; m0, m1 as in pair_x2_d.
__device__ __forceinline__ void pair_x2_dt(float2 dx, float2 dy, float2 dz, bool m0, bool m1, float rc2, float2 sg,
                                           float2 e24, float2 e4, float2 us, Acc2& c) {
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
  c.fx = __ffma2_rn(q, dx, c.fx);
  c.fy = __ffma2_rn(q, dy, c.fy);
  c.fz = __ffma2_rn(q, dz, c.fz);
  c.en = __fadd2_rn(c.en, __ffma2_rn(e4, __fmul2_rn(s6, __fadd2_rn(s6, m1f)), make_float2(-us.x, -us.y)));
  c.vir = __fadd2_rn(c.vir, pv);
  c.np += (int)a0 + (int)a1;
}

// Typed form of pair_range_x2 for one or two types.  k8 holds particle i's
// row: k8[t] the energy shift, k8[2 + t] sigma^2, k8[4 + t] 24 eps, k8[6 + t]
// 4 eps of the pair type (type of i, t); a candidate's type is 1 if its w is
// at least 1 (type_of clamped to two types), and with one type both columns
// are equal.
template <bool SJ>
__device__ __forceinline__ void pair_range_x2t(const float4* __restrict__ pos, int lo, int hi, float xi, float yi,
                                               float zi, float shx, float shy, float shz, float rc2,
                                               const float* k8, Acc2& c) {
  for (int j = lo; j < hi; j += 2) {
    const bool has1 = j + 1 < hi;
    const int j1 = has1 ? j + 1 : j;
    const float4 p0 = __ldg(pos + j), p1 = __ldg(pos + j1);
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
    pair_x2_dt(dx, dy, dz, true, has1, rc2, make_float2(t0 ? k8[3] : k8[2], t1 ? k8[3] : k8[2]),
               make_float2(t0 ? k8[5] : k8[4], t1 ? k8[5] : k8[4]), make_float2(t0 ? k8[7] : k8[6], t1 ? k8[7] : k8[6]),
               make_float2(t0 ? k8[1] : k8[0], t1 ? k8[1] : k8[0]), c);
  }
}

// STAGED: pos points into a shared-memory tile (plain loads) instead of
// global memory (read-only cached loads).
template <bool SJ, bool STAGED = false>
__device__ __forceinline__ void pair_range_x2(const float4* __restrict__ pos, int lo, int hi, float xi, float yi,
                                              float zi, float shx, float shy, float shz, float rc2, Acc2& c) {
  for (int j = lo; j < hi; j += 2) {
    const bool has1 = j + 1 < hi;
    const int j1 = has1 ? j + 1 : j;
    const float4 p0 = STAGED ? pos[j] : __ldg(pos + j), p1 = STAGED ? pos[j1] : __ldg(pos + j1);
    pair_x2<SJ>(p0, p1, true, has1, xi, yi, zi, shx, shy, shz, rc2, c);
  }
}

// Segment dispatch: the packed loop for FP32 (one type, or up to two types
// with the row constants in ushift[0 .. 7]), the scalar loop otherwise.
template <typename R, bool SJ, bool TYPED, bool X2>
__device__ __forceinline__ void segment(const typename RT<R>::R4* __restrict__ pos, int lo, int hi, R xi, R yi, R zi,
                                        R shx, R shy, R shz, R rc2, int ti, const ForceArgs<R>& a, const R* ushift,
                                        Acc<R>& c, Acc2& c2) {
  if constexpr (X2 && TYPED) {
    pair_range_x2t<SJ>(pos, lo, hi, xi, yi, zi, shx, shy, shz, rc2, ushift, c2);
  } else if constexpr (X2) {
    pair_range_x2<SJ>(pos, lo, hi, xi, yi, zi, shx, shy, shz, rc2, c2);
  } else {
    pair_range<R, SJ, TYPED>(pos, lo, hi, xi, yi, zi, shx, shy, shz, rc2, ti, a, ushift, c);
  }
}

// Which segments of the row walk are evaluated: all of them, or only those
// that reach a periodic image (a row outside the grid in y or z, or the part
// of a window beyond either x end).
enum class Walk { kAll, kImagesOnly };

// The culled cell-row walk of particle `self` (position pi, clamped cutoff
// rci) over the cell grid g whose cell starts are start[0 .. ncell] (positions
// pos sorted by cell), accumulating into c (scalar loop) or c2 (packed).
template <typename R, bool TYPED, bool X2, Walk MODE = Walk::kAll>
__device__ __forceinline__ void walk_rows(const typename RT<R>::R4* __restrict__ pos,
                                          const int32_t* __restrict__ start, const Grid<R>& g,
                                          const ForceArgs<R>& a, int self, const typename RT<R>::R4& pi, R rci,
                                          int ti, const R* ushift, Acc<R>& c, Acc2& c2) {
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
      const int64_t row = (int64_t)nx * (wy + (int64_t)ny * wz);
      // segment u < 0: image -L (shift j)
      if (ulo < 0) {
        int a1 = min(uhi, -1);
        int j0 = __ldg(start + row + ulo + nx), j1 = __ldg(start + row + a1 + nx + 1);
        segment<R, true, TYPED, X2>(pos, j0, j1, pi.x, yi, zi, -g.L[0], ysh, zsh, rc2, ti, a, ushift, c, c2);
      }
      // segment 0 <= u < nx: no x shift; the particle itself is skipped
      const bool img_row = uy < 0 || uy >= ny || uz < 0 || uz >= nz;
      if (!kImg || img_row) {
        int a0 = max(ulo, 0), a1 = min(uhi, nx - 1);
        if (a0 <= a1) {
          int j0 = __ldg(start + row + a0), j1 = __ldg(start + row + a1 + 1);
          if (!kImg && uy == cy && uz == cz) {  // the particle's own row: cut it out
            segment<R, false, TYPED, X2>(pos, j0, min(j1, self), pi.x, yi, zi, 0, 0, 0, rc2, ti, a, ushift, c, c2);
            segment<R, false, TYPED, X2>(pos, max(j0, self + 1), j1, pi.x, yi, zi, 0, 0, 0, rc2, ti, a, ushift, c,
                                         c2);
          } else if (ysh == (R)0 && zsh == (R)0) {
            segment<R, false, TYPED, X2>(pos, j0, j1, pi.x, yi, zi, 0, 0, 0, rc2, ti, a, ushift, c, c2);
          } else {
            segment<R, true, TYPED, X2>(pos, j0, j1, pi.x, yi, zi, (R)0, ysh, zsh, rc2, ti, a, ushift, c, c2);
          }
        }
      }
      // segment u >= nx: image +L (shift i)
      if (uhi >= nx) {
        int a0 = max(ulo, nx);
        int j0 = __ldg(start + row + a0 - nx), j1 = __ldg(start + row + uhi - nx + 1);
        segment<R, true, TYPED, X2>(pos, j0, j1, pi.x - g.L[0], yi, zi, (R)0, ysh, zsh, rc2, ti, a, ushift, c, c2);
      }
    }
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
// pos, sorted by cell).  Returns the force and writes e_i, w_i, pairs.
template <typename R, bool TYPED, bool X2 = false>
__device__ __forceinline__ typename RT<R>::R4 force_one(const typename RT<R>::R4* __restrict__ pos,
                                                        const int32_t* __restrict__ start, const Grid<R>& g,
                                                        const ForceArgs<R>& a, int self,
                                                        const typename RT<R>::R4& pi, R rc_in, R& e_out, R& w_out,
                                                        int& np_out) {
  static_assert(!X2 || sizeof(R) == 4, "the packed loop serves FP32 only (with types: at most two)");
  Acc<R> c;
  Acc2 c2;
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
  walk_rows<R, TYPED, X2>(pos, start, g, a, self, pi, rci, ti, ushift, c, c2);
  if constexpr (X2) {  // fold the two packed lanes (and the sign of d) into c
    c.fx = -(c2.fx.x + c2.fx.y);
    c.fy = -(c2.fy.x + c2.fy.y);
    c.fz = -(c2.fz.x + c2.fz.y);
    c.en = c2.en.x + c2.en.y;
    c.vir = c2.vir.x + c2.vir.y;
    c.np = c2.np;
  }
  typename RT<R>::R4 out;
  if (TYPED) {
    out.x = c.fx;
    out.y = c.fy;
    out.z = c.fz;
    e_out = (R)0.5 * c.en;
    w_out = (R)0.5 * c.vir;
  } else {
    out.x = (R)24 * c.fx;
    out.y = (R)24 * c.fy;
    out.z = (R)24 * c.fz;
    e_out = (R)2 * c.en - (R)0.5 * (R)c.np * ushift[0];
    w_out = (R)12 * c.vir;
  }
  out.w = e_out;
  np_out = c.np;
  return out;
}

}  // namespace dcm
