// Adjoint of the force/energy map (differentiation form): gradients of a
// scalar loss L(F, E) with respect to positions and per-type LJ parameters,
// with the per-particle cutoffs held fixed.
//
// For upstream A_i = dL/dF_i and dLdE = dL/dE, N(i) = {j != i : |r_ij| < rc_i}:
//   dL/dr_k = sum_{j in N(k)}       [ J(r_kj) A_k - dLdE/2 phi_kj ]
//           + sum_{j : k in N(j)}   [ -J(r_kj) A_j - dLdE/2 phi_kj ]
// phi_ij = g(r) r_ij is the force on i from j, J = g I + (g'/r) r r^T its
// (symmetric) Jacobian, g = 24 eps [2 s12 - s6] / r^2 and
// g'/r = 24 eps [-28 s12 + 8 s6] / r^4 with s6 = (sigma/r)^6, s12 = s6^2.
// Because the cutoffs differ per particle the second (reverse) sum runs over
// the j whose own cutoff reaches k: one thread per k walks the stencil of a
// radius that bounds every such rc_j, and every candidate is tested against
// both rc_k (forward pair) and rc_j (reverse pair).  The bound is the largest
// cutoff in the 27 blocks around k, blocks of edge at least 1.001 rc_max
// (a j with |r_kj| < rc_j <= rc_max lies in one of them), so away from the
// interfaces, where every cutoff is rc_min, the walk covers the rc_min
// sphere instead of the rc_max one.  The forward force itself is not
// needed: only A and dLdE enter.
//
// Parameter gradients per type pair p of every forward pair (k, j in N(k)):
//   dL/deps_p   += A_k . phi_kj / eps_p + dLdE/2 (U - U(rc_k) if shifted) / eps_p
//   dL/dsigma_p += A_k . (dg/dsigma) r_kj + dLdE/2 d(U - U(rc_k))/dsigma
// Both terms are eps_p (resp. eps_p / sigma_p) times a function of s6 alone:
//   d/deps:   24 (2 s12 - s6) / r^2 (A_k . r_kj) + 2 dLdE [(s12 - s6) - (c12 - c6)]
//   d/dsigma: 24 (24 s12 - 6 s6) / r^2 (A_k . r_kj) + 2 dLdE [(12 s12 - 6 s6) - (12 c12 - 6 c6)]
//             times eps_p / sigma_p
// with c6 = (sigma_p / rc_k)^6 when shifted (else the c terms are 0), so the
// pair loop sums the brackets (no division or root per pair) and the factor
// eps_p / sigma_p is applied once to each warp's sum.  The sums are taken per
// warp in the working precision, reduced in FP64, then chained to per-type
// gradients through Lorentz-Berthelot mixing.
#include <algorithm>

#include "forces_core.cuh"
#include "tile_order.cuh"

namespace dcm {

// Blocks of the reverse-pair bound: nb[d] per axis of edge L[d] / nb[d].
struct BlockGrid {
  int nb[3];
  float inv_be[3];
};

__device__ __forceinline__ int block_coord(float x, float inv_be, int nb) {
  return (int)fminf(fmaxf(floorf(x * inv_be), 0.f), (float)(nb - 1));  // NaN -> 0
}

__device__ __forceinline__ float up_float(float v) { return v; }
__device__ __forceinline__ float up_float(double v) { return __double2float_ru(v); }

// Largest cutoff of each block (float bits: the order of positive floats is
// the order of their bit patterns), rounded up from FP64.
template <typename R>
__global__ void k_block_max(int64_t n, const typename RT<R>::R4* __restrict__ pos, const R* __restrict__ rc,
                            R rc_max, BlockGrid bg, int32_t* __restrict__ bmax) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto p = ldg4(pos + i);
  R v = rc[i];
  if (!(v <= rc_max)) v = rc_max;
  if (!(v > (R)0)) v = (R)0;
  const int bx = block_coord((float)p.x, bg.inv_be[0], bg.nb[0]);
  const int by = block_coord((float)p.y, bg.inv_be[1], bg.nb[1]);
  const int bz = block_coord((float)p.z, bg.inv_be[2], bg.nb[2]);
  atomicMax(bmax + bx + bg.nb[0] * (by + bg.nb[1] * bz), __float_as_int(up_float(v)));
}

template <typename R>
struct AdjAcc {
  R gx = 0, gy = 0, gz = 0;
  R de[16], ds[16];  // per type pair (only [0] for one type)
};

template <typename R, bool TYPED>
__device__ __forceinline__ void adj_range(const typename RT<R>::R4* __restrict__ pos, const R* __restrict__ rc,
                                          const typename RT<R>::R4* __restrict__ A, int lo, int hi, int self, R xi,
                                          R yi, R zi, R shx, R shy, R shz, R rck2, int tk,
                                          const typename RT<R>::R4& ak, R half_dlde, const ForceArgs<R>& a,
                                          const R* ku, const R* kd, AdjAcc<R>& c) {
  for (int j = lo; j < hi; ++j) {
    if (j == self) continue;
    auto pj = ldg4(pos + j);
    R dx = xi - (pj.x + shx);
    R dy = yi - (pj.y + shy);
    R dz = zi - (pj.z + shz);
    R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    R rcj = rc[j];
    if (!(rcj <= a.rc_max)) rcj = a.rc_max;
    bool fwd = r2 < rck2;
    bool rev = r2 < rcj * rcj;
    if (!(fwd || rev)) continue;
    int tj = TYPED ? type_of(pj.w, a.ntypes) : 0;
    int p = TYPED ? tk * a.ntypes + tj : 0;
    R e24 = TYPED ? a.eps24[p] : (R)24;
    R sig2 = TYPED ? a.sig2[p] : (R)1;
    R inv = recip(r2);
    R s2 = sig2 * inv;
    R s6 = s2 * s2 * s2, s12 = s6 * s6;
    R g = e24 * ((R)2 * s12 - s6) * inv;
    R gpr = e24 * ((R)-28 * s12 + (R)8 * s6) * inv * inv;
    R ex = -half_dlde * g;  // -dLdE/2 phi / r_vec, both sums
    R tx = 0, ty = 0, tz = 0;
    if (fwd) {
      R ra = dx * ak.x + dy * ak.y + dz * ak.z;
      tx += g * ak.x + gpr * ra * dx;
      ty += g * ak.y + gpr * ra * dy;
      tz += g * ak.z + gpr * ra * dz;
      tx += ex * dx;
      ty += ex * dy;
      tz += ex * dz;
      R cu = TYPED ? (tj == 0 ? ku[0] : tj == 1 ? ku[1] : tj == 2 ? ku[2] : ku[3]) : ku[0];
      R cd = TYPED ? (tj == 0 ? kd[0] : tj == 1 ? kd[1] : tj == 2 ? kd[2] : kd[3]) : kd[0];
      R hd2 = (R)4 * half_dlde;
      c.de[p] += (R)24 * ((R)2 * s12 - s6) * inv * ra + hd2 * ((s12 - s6) - cu);
      c.ds[p] += (R)24 * ((R)24 * s12 - (R)6 * s6) * inv * ra + hd2 * (((R)12 * s12 - (R)6 * s6) - cd);
    }
    if (rev) {
      auto aj = ldg4(A + j);
      R ra = dx * aj.x + dy * aj.y + dz * aj.z;
      tx -= g * aj.x + gpr * ra * dx;
      ty -= g * aj.y + gpr * ra * dy;
      tz -= g * aj.z + gpr * ra * dz;
      tx += ex * dx;
      ty += ex * dy;
      tz += ex * dz;
    }
    c.gx += tx;
    c.gy += ty;
    c.gz += tz;
  }
}

// The culled row walk of the adjoint (radius `reach`, the reverse pairs'
// bound) around the particle `self` at pi, handing each row segment to
// range(lo, hi, self_or_-1, xi, yi, zi, shx, shy, shz) as the force walk does
// (image segments with the exact shifts; self is passed only for the
// particle's own image, where it must be skipped).
template <typename R, typename F>
__device__ __forceinline__ void adj_walk(const int32_t* __restrict__ start, const Grid<R>& g,
                                         const typename RT<R>::R4& pi, R reach2s, R reach, int self, F&& range) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const R l = g.edge, il = g.inv_edge, ilx = g.inv_edge_x;
  const int cx = cell_coord<R>(pi.x, g.edge_x, ilx, nx);
  const int cy = cell_coord<R>(pi.y, l, il, ny);
  const int cz = cell_coord<R>(pi.z, l, il, nz);
  const int H = (int)ceil(reach * il), Hx = (int)ceil(reach * ilx);
  for (int uz = cz - H; uz <= cz + H; ++uz) {
    R gz = uz > cz ? (R)uz * l - pi.z : (uz < cz ? pi.z - (R)(uz + 1) * l : (R)0);
    R gz2 = gz * gz;
    if (gz2 >= reach2s) continue;
    int wz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
    R zi = uz >= nz ? pi.z - g.L[2] : pi.z;
    R zsh = uz < 0 ? -g.L[2] : (R)0;
    for (int uy = cy - H; uy <= cy + H; ++uy) {
      R gy = uy > cy ? (R)uy * l - pi.y : (uy < cy ? pi.y - (R)(uy + 1) * l : (R)0);
      R gyz2 = gz2 + gy * gy;
      if (gyz2 >= reach2s) continue;
      int wy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
      R yi = uy >= ny ? pi.y - g.L[1] : pi.y;
      R ysh = uy < 0 ? -g.L[1] : (R)0;
      R wx = sqrt(reach2s - gyz2);
      int ulo = ufloor<R>((pi.x - wx) * ilx - (R)5e-4);
      int uhi = ufloor<R>((pi.x + wx) * ilx + (R)5e-4);
      ulo = max(ulo, cx - Hx);
      uhi = min(uhi, cx + Hx);
      if (ulo > uhi) continue;  // a coordinate outside [0, L): no window
      const int64_t row = (int64_t)nx * (wy + (int64_t)ny * wz);
      if (ulo < 0) {
        int a1 = min(uhi, -1);
        range(__ldg(start + row + ulo + nx), __ldg(start + row + a1 + nx + 1), -1, pi.x, yi, zi, -g.L[0], ysh, zsh);
      }
      {
        int a0 = max(ulo, 0), a1 = min(uhi, nx - 1);
        if (a0 <= a1)
          range(__ldg(start + row + a0), __ldg(start + row + a1 + 1), (ysh == (R)0 && zsh == (R)0) ? self : -1, pi.x,
                yi, zi, (R)0, ysh, zsh);
      }
      if (uhi >= nx) {
        int a0 = max(ulo, nx);
        range(__ldg(start + row + a0 - nx), __ldg(start + row + uhi - nx + 1), -1, pi.x - g.L[0], yi, zi, (R)0, ysh,
              zsh);
      }
    }
  }
}

// The same walk split in two for the packed adjoint: in every row the cells
// within the particle's own cutoff rk (the inner window: forward and reverse
// pairs) go to full(lo, hi, self, xi, yi, zi, shx, shy, shz) and the rest of
// the window of radius `reach` (the shell: only pairs with rc_j > r >= rk,
// rare away from the interfaces) to shell(...).  Pieces are split at the
// periodic x boundary as in adj_walk.
template <typename R, typename F, typename S>
__device__ __forceinline__ void adj_walk2(const int32_t* __restrict__ start, const Grid<R>& g,
                                          const typename RT<R>::R4& pi, R rk, R reach, int self, F&& full,
                                          S&& shell) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const R l = g.edge, il = g.inv_edge, ilx = g.inv_edge_x;
  const R reach2s = reach * reach * (R)1.000004, rk2s = rk * rk * (R)1.000004;
  const int cx = cell_coord<R>(pi.x, g.edge_x, ilx, nx);
  const int cy = cell_coord<R>(pi.y, l, il, ny);
  const int cz = cell_coord<R>(pi.z, l, il, nz);
  const int H = (int)ceil(reach * il), Hx = (int)ceil(reach * ilx);
  for (int uz = cz - H; uz <= cz + H; ++uz) {
    R gz = uz > cz ? (R)uz * l - pi.z : (uz < cz ? pi.z - (R)(uz + 1) * l : (R)0);
    R gz2 = gz * gz;
    if (gz2 >= reach2s) continue;
    int wz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
    R zi = uz >= nz ? pi.z - g.L[2] : pi.z;
    R zsh = uz < 0 ? -g.L[2] : (R)0;
    for (int uy = cy - H; uy <= cy + H; ++uy) {
      R gy = uy > cy ? (R)uy * l - pi.y : (uy < cy ? pi.y - (R)(uy + 1) * l : (R)0);
      R gyz2 = gz2 + gy * gy;
      if (gyz2 >= reach2s) continue;
      int wy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
      R yi = uy >= ny ? pi.y - g.L[1] : pi.y;
      R ysh = uy < 0 ? -g.L[1] : (R)0;
      R wx = sqrt(reach2s - gyz2);
      int ulo = max(ufloor<R>((pi.x - wx) * ilx - (R)5e-4), cx - Hx);
      int uhi = min(ufloor<R>((pi.x + wx) * ilx + (R)5e-4), cx + Hx);
      if (ulo > uhi) continue;  // a coordinate outside [0, L): no window
      int ilo = uhi + 1, ihi = uhi;  // inner window (empty unless the row meets the rk sphere)
      if (gyz2 < rk2s) {
        R wi = sqrt(rk2s - gyz2);
        ilo = min(max(ufloor<R>((pi.x - wi) * ilx - (R)5e-4), ulo), uhi + 1);
        ihi = max(min(ufloor<R>((pi.x + wi) * ilx + (R)5e-4), uhi), ilo - 1);
      }
      const int64_t row = (int64_t)nx * (wy + (int64_t)ny * wz);
      const bool same = ysh == (R)0 && zsh == (R)0;
      // cells [u0, u1] of the unwrapped row, split at the x boundary
      auto emit = [&](int u0, int u1, bool inner) {
        if (u0 > u1) return;
        if (u0 < 0) {
          const int a1 = min(u1, -1);
          const int j0 = __ldg(start + row + u0 + nx), j1 = __ldg(start + row + a1 + nx + 1);
          if (inner) full(j0, j1, -1, pi.x, yi, zi, -g.L[0], ysh, zsh);
          else shell(j0, j1, -1, pi.x, yi, zi, -g.L[0], ysh, zsh);
        }
        const int a0 = max(u0, 0), a1 = min(u1, nx - 1);
        if (a0 <= a1) {
          const int j0 = __ldg(start + row + a0), j1 = __ldg(start + row + a1 + 1);
          if (inner) full(j0, j1, same ? self : -1, pi.x, yi, zi, (R)0, ysh, zsh);
          else shell(j0, j1, same ? self : -1, pi.x, yi, zi, (R)0, ysh, zsh);
        }
        if (u1 >= nx) {
          const int b0 = max(u0, nx);
          const int j0 = __ldg(start + row + b0 - nx), j1 = __ldg(start + row + u1 - nx + 1);
          if (inner) full(j0, j1, -1, pi.x - g.L[0], yi, zi, (R)0, ysh, zsh);
          else shell(j0, j1, -1, pi.x - g.L[0], yi, zi, (R)0, ysh, zsh);
        }
      };
      emit(ulo, ilo - 1, false);
      emit(ilo, ihi, true);
      emit(ihi + 1, uhi, false);
    }
  }
}

// Radius of the adjoint walk of particle k: the largest cutoff in the 27
// blocks around it (every j whose own cutoff reaches k lies in one of them),
// at least rc_k; rc_max without the block table.
template <typename R>
__device__ __forceinline__ R reverse_reach(const typename RT<R>::R4& pi, R rck, R rc_max, const BlockGrid& bg,
                                           const int32_t* __restrict__ bmax) {
  R reach = rc_max;
  if (bmax) {
    const int bx = block_coord((float)pi.x, bg.inv_be[0], bg.nb[0]);
    const int by = block_coord((float)pi.y, bg.inv_be[1], bg.nb[1]);
    const int bz = block_coord((float)pi.z, bg.inv_be[2], bg.nb[2]);
    float m = 0.f;
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = (bz + dz + bg.nb[2]) % bg.nb[2];
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = (by + dy + bg.nb[1]) % bg.nb[1];
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = (bx + dx + bg.nb[0]) % bg.nb[0];
          m = fmaxf(m, __int_as_float(__ldg(bmax + xx + bg.nb[0] * (yy + bg.nb[1] * zz))));
        }
      }
    }
    reach = (R)m < reach ? (R)m : reach;
    if (reach < rck) reach = rck;
  }
  return reach;
}

// Threads per block of the adjoint: the cost per particle varies several-fold
// (rc_k and the reverse reach grow toward the interfaces), so small blocks
// free their slots as soon as their own warps finish (measured best: 64 for
// FP32, 32 for FP64).
template <typename R>
constexpr int adj_block() {
  return sizeof(R) == 4 ? 64 : 32;
}

template <typename R, bool TYPED>
__global__ void __launch_bounds__(adj_block<R>()) k_adjoint(int64_t n, const typename RT<R>::R4* __restrict__ pos,
                                                            const R* __restrict__ rc, const int32_t* __restrict__ start,
                                                            ForceArgs<R> a, const typename RT<R>::R4* __restrict__ A,
                                                            R half_dlde, typename RT<R>::R4* __restrict__ G,
                                                            double* __restrict__ part, int64_t nwarp, BlockGrid bg,
                                                            const int32_t* __restrict__ bmax,
                                                            const int32_t* __restrict__ order) {
  const int64_t i = (int64_t)(order ? __ldg(order + blockIdx.x) : (int32_t)blockIdx.x) * blockDim.x + threadIdx.x;
  const int np = a.ntypes * a.ntypes;
  AdjAcc<R> c;
  for (int p = 0; p < 16; ++p) c.de[p] = c.ds[p] = (R)0;
  if (i < n) {
    const Grid<R>& g = a.g;
    auto pi = ldg4(pos + i);
    auto ak = ldg4(A + i);
    R rck = rc[i];
    if (!(rck <= a.rc_max)) rck = a.rc_max;
    if (!(rck > (R)0)) rck = (R)0;
    const R rck2 = rck * rck;
    const R reach = reverse_reach<R>(pi, rck, a.rc_max, bg, bmax);
    const R reach2s = reach * reach * (R)1.000004;
    const int tk = TYPED ? type_of(pi.w, a.ntypes) : 0;
    // (sigma_p / rc_k)^6 terms of the shifted energy per partner type
    R ku[4] = {0, 0, 0, 0}, kd[4] = {0, 0, 0, 0};
    if (a.shift) {
      for (int t = 0; t < (TYPED ? a.ntypes : 1); ++t) {
        R sig2 = TYPED ? a.sig2[tk * a.ntypes + t] : (R)1;
        R c2 = sig2 / rck2, c6 = c2 * c2 * c2, c12 = c6 * c6;
        ku[t] = c12 - c6;
        kd[t] = (R)12 * c12 - (R)6 * c6;
      }
    }
    adj_walk<R>(start, g, pi, reach2s, reach, (int)i,
                [&](int lo, int hi, int self, R xi, R yi, R zi, R shx, R shy, R shz) {
                  adj_range<R, TYPED>(pos, rc, A, lo, hi, self, xi, yi, zi, shx, shy, shz, rck2, tk, ak, half_dlde, a,
                                      ku, kd, c);
                });
    typename RT<R>::R4 out;
    out.x = c.gx;
    out.y = c.gy;
    out.z = c.gz;
    out.w = (R)0;
    G[i] = out;
  }
  if (part) {
    int64_t w = i >> 5;
    for (int p = 0; p < np; ++p) {
      R de = c.de[p], ds = c.ds[p];
      for (int o = 16; o > 0; o >>= 1) {
        de += __shfl_xor_sync(0xffffffffu, de, o);
        ds += __shfl_xor_sync(0xffffffffu, ds, o);
      }
      if ((threadIdx.x & 31) == 0) {
        // eps_p / sigma_p, the factor taken out of the d/dsigma terms
        const double f = TYPED ? 0.25 * (double)a.eps4[p] / sqrt((double)a.sig2[p]) : 1.0;
        part[(int64_t)p * nwarp + w] = (double)de;
        part[(int64_t)(16 + p) * nwarp + w] = (double)ds * f;
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Packed form (FP32, one or two types): candidates j and j + 1 of a segment in
// one FP32x2 step, branch-free (a slot that is neither a forward nor a reverse
// pair gets 1/r^2 = 0, which zeroes its terms), the parameter sums per partner
// type in registers.  With d = r_j - r_k = -r_kj the terms read
//   G_k += fwd [g A_k + g'/r (d.A_k) d] - rev [g A_j + g'/r (d.A_j) d]
//          + (fwd + rev) dLdE/2 g d,
//   de_t += fwd [24 (2 s12 - s6) y (-d.A_k) + 2 dLdE ((s12 - s6) - cu_t)],
//   ds_t += fwd [24 (24 s12 - 6 s6) y (-d.A_k) + 2 dLdE ((12 s12 - 6 s6) - cd_t)],
// y = 1/r^2 (refined as in the force loop), t the partner's type.
// ----------------------------------------------------------------------------
struct AdjAcc2 {
  float2 gx = {0.f, 0.f}, gy = {0.f, 0.f}, gz = {0.f, 0.f};
  float2 de[2] = {{0.f, 0.f}, {0.f, 0.f}}, ds[2] = {{0.f, 0.f}, {0.f, 0.f}};
};

// Particle k's constants for partner type t in {0, 1}: sigma^2, 24 eps of the
// pair type, and the shifted-energy terms cu, cd.
struct AdjRow {
  float sg[2], e24[2], cu[2], cd[2];
};

template <bool SJ>
__device__ __forceinline__ void adj_range_x2(const float4* __restrict__ pos, const float* __restrict__ rc,
                                             const float4* __restrict__ A, int lo, int hi, int self, float xi,
                                             float yi, float zi, float shx, float shy, float shz, float rck2,
                                             float rc_max, const float4& ak, float half_dlde, const AdjRow& k,
                                             AdjAcc2& c) {
  const float2 two = make_float2(2.f, 2.f), m1 = make_float2(-1.f, -1.f), one = make_float2(1.f, 1.f);
  const float2 akx = make_float2(ak.x, ak.x), aky = make_float2(ak.y, ak.y), akz = make_float2(ak.z, ak.z);
  const float hd2 = 4.f * half_dlde;
  for (int j = lo; j < hi; j += 2) {
    const bool has1 = j + 1 < hi;
    const int j1 = has1 ? j + 1 : j;
    const float4 p0 = __ldg(pos + j), p1 = __ldg(pos + j1);
    const float4 a0 = __ldg(A + j), a1 = __ldg(A + j1);
    const float rc0 = clamp_cutoff<float>(__ldg(rc + j), rc_max), rc1 = clamp_cutoff<float>(__ldg(rc + j1), rc_max);
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
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    const bool v0 = j != self, v1 = has1 && j1 != self;
    const bool f0 = v0 && r2.x < rck2, f1 = v1 && r2.y < rck2;
    const bool b0 = v0 && r2.x < rc0 * rc0, b1 = v1 && r2.y < rc1 * rc1;
    float y0, y1;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(r2.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(r2.y));
    float2 y = make_float2(y0, y1);
    const float2 e = __ffma2_rn(make_float2(-r2.x, -r2.y), y, one);
    y = __ffma2_rn(y, e, y);
    y = make_float2(f0 || b0 ? y.x : 0.f, f1 || b1 ? y.y : 0.f);
    const bool t0 = p0.w >= 1.f, t1 = p1.w >= 1.f;
    const float2 sg = make_float2(t0 ? k.sg[1] : k.sg[0], t1 ? k.sg[1] : k.sg[0]);
    const float2 e24 = make_float2(t0 ? k.e24[1] : k.e24[0], t1 ? k.e24[1] : k.e24[0]);
    const float2 s2 = __fmul2_rn(sg, y);
    const float2 s6 = __fmul2_rn(__fmul2_rn(s2, s2), s2), s12 = __fmul2_rn(s6, s6);
    const float2 ey = __fmul2_rn(e24, y);
    const float2 g = __fmul2_rn(ey, __ffma2_rn(two, s12, make_float2(-s6.x, -s6.y)));        // 24 eps (2 s12 - s6) / r^2
    const float2 gp = __fmul2_rn(__fmul2_rn(ey, y),
                                 __ffma2_rn(make_float2(-28.f, -28.f), s12, __fmul2_rn(make_float2(8.f, 8.f), s6)));
    const float2 fw = make_float2(f0 ? 1.f : 0.f, f1 ? 1.f : 0.f), rv = make_float2(b0 ? 1.f : 0.f, b1 ? 1.f : 0.f);
    const float2 dak = __ffma2_rn(dx, akx, __ffma2_rn(dy, aky, __fmul2_rn(dz, akz)));
    const float2 ajx = make_float2(a0.x, a1.x), ajy = make_float2(a0.y, a1.y), ajz = make_float2(a0.z, a1.z);
    const float2 daj = __ffma2_rn(dx, ajx, __ffma2_rn(dy, ajy, __fmul2_rn(dz, ajz)));
    const float2 gf = __fmul2_rn(g, fw), gr = __fmul2_rn(g, rv);
    // coefficient of d: g'/r (fwd d.A_k - rev d.A_j) + (fwd + rev) dLdE/2 g
    const float2 cd = __ffma2_rn(gp, __ffma2_rn(fw, dak, __fmul2_rn(make_float2(-rv.x, -rv.y), daj)),
                                 __fmul2_rn(__fadd2_rn(fw, rv), __fmul2_rn(make_float2(half_dlde, half_dlde), g)));
    c.gx = __fadd2_rn(c.gx, __ffma2_rn(cd, dx, __ffma2_rn(gf, akx, __fmul2_rn(make_float2(-gr.x, -gr.y), ajx))));
    c.gy = __fadd2_rn(c.gy, __ffma2_rn(cd, dy, __ffma2_rn(gf, aky, __fmul2_rn(make_float2(-gr.x, -gr.y), ajy))));
    c.gz = __fadd2_rn(c.gz, __ffma2_rn(cd, dz, __ffma2_rn(gf, akz, __fmul2_rn(make_float2(-gr.x, -gr.y), ajz))));
    // parameter sums of the forward pairs, by partner type
    const float2 rfa = __fmul2_rn(__fmul2_rn(y, make_float2(-dak.x, -dak.y)), make_float2(24.f, 24.f));  // 24 y (r.A_k)
    const float2 ue = __fadd2_rn(s12, make_float2(-s6.x, -s6.y));                                      // s12 - s6
    const float2 us = __ffma2_rn(make_float2(12.f, 12.f), s12, __fmul2_rn(make_float2(-6.f, -6.f), s6));
    const float2 cu = make_float2(t0 ? k.cu[1] : k.cu[0], t1 ? k.cu[1] : k.cu[0]);
    const float2 cdd = make_float2(t0 ? k.cd[1] : k.cd[0], t1 ? k.cd[1] : k.cd[0]);
    const float2 hd = make_float2(hd2, hd2);
    const float2 te = __fmul2_rn(fw, __ffma2_rn(rfa, __ffma2_rn(two, s12, make_float2(-s6.x, -s6.y)),
                                                __fmul2_rn(hd, __fadd2_rn(ue, make_float2(-cu.x, -cu.y)))));
    const float2 u24 = __ffma2_rn(make_float2(24.f, 24.f), s12, __fmul2_rn(make_float2(-6.f, -6.f), s6));
    const float2 ts = __fmul2_rn(fw, __ffma2_rn(rfa, u24, __fmul2_rn(hd, __fadd2_rn(us, make_float2(-cdd.x, -cdd.y)))));
    // slot a of the packed pair belongs to partner type t_a
    c.de[0] = __fadd2_rn(c.de[0], make_float2(t0 ? 0.f : te.x, t1 ? 0.f : te.y));
    c.de[1] = __fadd2_rn(c.de[1], make_float2(t0 ? te.x : 0.f, t1 ? te.y : 0.f));
    c.ds[0] = __fadd2_rn(c.ds[0], make_float2(t0 ? 0.f : ts.x, t1 ? 0.f : ts.y));
    c.ds[1] = __fadd2_rn(c.ds[1], make_float2(t0 ? ts.x : 0.f, t1 ? ts.y : 0.f));
  }
}

// Shell candidates of the packed adjoint: r >= rc_k up to cell rounding, so
// the forward test fails for nearly all of them and the reverse test
// (r < rc_j) rarely passes; each candidate costs a distance test, and the
// few pairs that pass either test take the scalar terms of adj_range.
__device__ __forceinline__ void adj_shell(const float4* __restrict__ pos, const float* __restrict__ rc,
                                          const float4* __restrict__ A, int lo, int hi, int self, float xi, float yi,
                                          float zi, float shx, float shy, float shz, float rck2, float rc_max,
                                          const float4& ak, float half_dlde, const AdjRow& k, AdjAcc2& c) {
  for (int j = lo; j < hi; ++j) {
    const float4 pj = __ldg(pos + j);
    const float dx = (pj.x + shx) - xi, dy = (pj.y + shy) - yi, dz = (pj.z + shz) - zi;  // d = r_j - r_k
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rcj = clamp_cutoff<float>(__ldg(rc + j), rc_max);
    const bool fwd = r2 < rck2 && j != self, rev = r2 < rcj * rcj && j != self;
    if (!(fwd || rev)) continue;
    const float4 aj = __ldg(A + j);
    const bool t = pj.w >= 1.f;
    const float y = recip(r2);
    const float s2 = (t ? k.sg[1] : k.sg[0]) * y, s6 = s2 * s2 * s2, s12 = s6 * s6;
    const float ey = (t ? k.e24[1] : k.e24[0]) * y;
    const float g = ey * fmaf(2.f, s12, -s6), gp = ey * y * fmaf(-28.f, s12, 8.f * s6);
    const float dak = fmaf(dx, ak.x, fmaf(dy, ak.y, dz * ak.z)), daj = fmaf(dx, aj.x, fmaf(dy, aj.y, dz * aj.z));
    const float fw = fwd ? 1.f : 0.f, rv = rev ? 1.f : 0.f;
    const float cd = gp * (fw * dak - rv * daj) + (fw + rv) * half_dlde * g;
    c.gx.x += cd * dx + fw * g * ak.x - rv * g * aj.x;
    c.gy.x += cd * dy + fw * g * ak.y - rv * g * aj.y;
    c.gz.x += cd * dz + fw * g * ak.z - rv * g * aj.z;
    if (fwd) {
      const float rfa = 24.f * y * -dak, hd2 = 4.f * half_dlde, us = 12.f * s12 - 6.f * s6;
      const float te = rfa * fmaf(2.f, s12, -s6) + hd2 * ((s12 - s6) - (t ? k.cu[1] : k.cu[0]));
      const float ts = rfa * (24.f * s12 - 6.f * s6) + hd2 * (us - (t ? k.cd[1] : k.cd[0]));
      if (t) {
        c.de[1].x += te;
        c.ds[1].x += ts;
      } else {
        c.de[0].x += te;
        c.ds[0].x += ts;
      }
    }
  }
}

constexpr int kAdjX2Block = 64;

__global__ void __launch_bounds__(kAdjX2Block) k_adjoint_x2(int64_t n, const float4* __restrict__ pos,
                                                            const float* __restrict__ rc,
                                                            const int32_t* __restrict__ start, ForceArgs<float> a,
                                                            const float4* __restrict__ A, float half_dlde,
                                                            float4* __restrict__ G, double* __restrict__ part,
                                                            int64_t nwarp, BlockGrid bg,
                                                            const int32_t* __restrict__ bmax,
                                                            const int32_t* __restrict__ order) {
  const int64_t i = (int64_t)(order ? __ldg(order + blockIdx.x) : (int32_t)blockIdx.x) * blockDim.x + threadIdx.x;
  const int nt = a.ntypes;
  AdjAcc2 c;
  int tk = 0;
  if (i < n) {
    const float4 pi = __ldg(pos + i);
    const float4 ak = __ldg(A + i);
    const float rck = clamp_cutoff<float>(__ldg(rc + i), a.rc_max), rck2 = rck * rck;
    const float reach = reverse_reach<float>(pi, rck, a.rc_max, bg, bmax);
    tk = type_of(pi.w, nt);
    AdjRow k;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int tc = t < nt ? t : nt - 1, p = tk * nt + tc;
      k.sg[t] = a.sig2[p];
      k.e24[t] = a.eps24[p];
      k.cu[t] = k.cd[t] = 0.f;
      if (a.shift && rck2 > 0.f) {
        const float c2 = a.sig2[p] / rck2, c6 = c2 * c2 * c2, c12 = c6 * c6;
        k.cu[t] = c12 - c6;
        k.cd[t] = 12.f * c12 - 6.f * c6;
      }
    }
    adj_walk2<float>(
        start, a.g, pi, rck, reach, (int)i,
        [&](int lo, int hi, int self, float xi, float yi, float zi, float shx, float shy, float shz) {
          if (shx == 0.f && shy == 0.f && shz == 0.f)
            adj_range_x2<false>(pos, rc, A, lo, hi, self, xi, yi, zi, shx, shy, shz, rck2, a.rc_max, ak, half_dlde,
                                k, c);
          else
            adj_range_x2<true>(pos, rc, A, lo, hi, self, xi, yi, zi, shx, shy, shz, rck2, a.rc_max, ak, half_dlde, k,
                               c);
        },
        [&](int lo, int hi, int self, float xi, float yi, float zi, float shx, float shy, float shz) {
          adj_shell(pos, rc, A, lo, hi, self, xi, yi, zi, shx, shy, shz, rck2, a.rc_max, ak, half_dlde, k, c);
        });
    G[i] = make_float4(c.gx.x + c.gx.y, c.gy.x + c.gy.y, c.gz.x + c.gz.y, 0.f);
  }
  if (part) {
    const int64_t w = i >> 5;
    for (int p = 0; p < nt * nt; ++p) {
      const bool mine = i < n && tk == p / nt, t1 = p % nt == 1;
      const float2 de2 = t1 ? c.de[1] : c.de[0], ds2 = t1 ? c.ds[1] : c.ds[0];
      float de = mine ? de2.x + de2.y : 0.f, ds = mine ? ds2.x + ds2.y : 0.f;
      for (int o = 16; o > 0; o >>= 1) {
        de += __shfl_xor_sync(0xffffffffu, de, o);
        ds += __shfl_xor_sync(0xffffffffu, ds, o);
      }
      if ((threadIdx.x & 31) == 0) {
        const double f = 0.25 * (double)a.eps4[p] / sqrt((double)a.sig2[p]);  // eps_p / sigma_p
        part[(int64_t)p * nwarp + w] = (double)de;
        part[(int64_t)(16 + p) * nwarp + w] = (double)ds * f;
      }
    }
  }
}

// Cost key of the adjoint's tiles (tile_order.cuh): the largest reverse reach
// among a tile's particles, the radius of its widest walk.
template <typename R>
__global__ void k_adj_tile_key(int64_t n, const typename RT<R>::R4* __restrict__ pos, const R* __restrict__ rc,
                               R rc_max, BlockGrid bg, const int32_t* __restrict__ bmax, int32_t* __restrict__ key,
                               int32_t* __restrict__ cnt, int64_t nchunk) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float r = 0.f;
  if (i < n) {
    const auto p = ldg4(pos + i);
    r = (float)reverse_reach<R>(p, clamp_cutoff<R>(rc[i], rc_max), rc_max, bg, bmax);
  }
  tile_key_of_block(r, (float)rc_max, key, cnt, nchunk);
}

// Per-type gradients from per-type-pair sums: eps_ab = sqrt(eps_a eps_b),
// sigma_ab = (sigma_a + sigma_b) / 2.  pair_de/ds: [ntypes^2]; out: [2 ntypes].
__global__ void k_mix_chain(const double* pair_de, const double* pair_ds, int nt, const double* eps, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int a = 0; a < 2 * nt; ++a) out[a] = 0.0;
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      int p = a * nt + b;
      if (a == b) {
        out[a] += pair_de[p];
        out[nt + a] += pair_ds[p];
      } else {
        out[a] += pair_de[p] * 0.5 * sqrt(eps[b] / eps[a]);
        out[b] += pair_de[p] * 0.5 * sqrt(eps[a] / eps[b]);
        out[nt + a] += 0.5 * pair_ds[p];
        out[nt + b] += 0.5 * pair_ds[p];
      }
    }
}

template <typename R>
int lj_adjoint(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc, const int32_t* cell_start,
               const typename RT<R>::R4* A, double dlde, typename RT<R>::R4* G, double* dparams, cudaStream_t st) {
  LJTable t = lj_table(ctx->p);
  int nt = t.ntypes;
  if (n <= 0) {
    if (dparams) DCM_CUDA_TRY(ctx, cudaMemsetAsync(dparams, 0, sizeof(double) * 2 * nt, st));
    return DCM_OK;
  }
  ForceArgs<R> a;
  a.g = cell_grid<R>(ctx);
  a.ntypes = nt;
  for (int k = 0; k < 16; ++k) {
    a.eps24[k] = (R)t.deps24[k];
    a.eps4[k] = (R)t.deps4[k];
    a.sig2[k] = (R)t.dsig2[k];
  }
  a.shift = ctx->p.shift_energy;
  a.rc_max = (R)ctx->p.rc_max;
  constexpr int kBlock = adj_block<R>();
  int64_t nblk = (n + kBlock - 1) / kBlock, nwarp = nblk * (kBlock / 32);
  bool want = dparams != nullptr;
  if (want && nwarp > ctx->red_cap)
    return set_error(ctx, DCM_ERR_CAPACITY, "adjoint reduction needs %lld partials", (long long)nwarp);
  double* part = want ? ctx->adj_part : nullptr;  // [32][nwarp]: de pairs 0..15, ds pairs 16..31
  BlockGrid bg;
  for (int d = 0; d < 3; ++d) {
    bg.nb[d] = ctx->nblk3[d];
    bg.inv_be[d] = (float)((double)ctx->nblk3[d] / ctx->p.box[d]);
  }
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->blk_max, 0, sizeof(int32_t) * ctx->nblk, st));
  DCM_LAUNCH(ctx, k_block_max<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, pos, rc, a.rc_max, bg, ctx->blk_max);
  // the packed loop (FP32, one or two types), else the scalar loop
  const bool x2 = sizeof(R) == 4 && nt <= 2;
  const int tb = x2 ? kAdjX2Block : kBlock;
  const void* kern = x2 ? (const void*)k_adjoint_x2
                        : (lj_general(t) ? (const void*)k_adjoint<R, true> : (const void*)k_adjoint<R, false>);
  static_assert(kAdjX2Block == adj_block<float>(), "the partials layout assumes equal blocks");
  // launch order of the tiles, the widest walks first, where that pays
  const TileOrder to = tile_order_layout(ctx->tile_scratch, (n + tb - 1) / tb);
  const int32_t* order = nullptr;
  if (tile_order_pays(kern, tb, to.ntile)) {
    int r0 = tile_order_begin(ctx, to, st);
    if (r0) return r0;
    DCM_LAUNCH(ctx, k_adj_tile_key<R>, (unsigned)to.ntile, tb, 0, st, n, pos, rc, a.rc_max, bg,
               (const int32_t*)ctx->blk_max, to.key, to.cnt, to.nchunk);
    if ((r0 = tile_order_finish(ctx, to, st))) return r0;
    order = to.order;
  }
  if constexpr (sizeof(R) == 4) {
    if (x2)
      DCM_LAUNCH(ctx, k_adjoint_x2, (unsigned)to.ntile, kAdjX2Block, 0, st, n, pos, rc, cell_start, a, A,
                 (float)(0.5 * dlde), G, part, nwarp, bg, (const int32_t*)ctx->blk_max, order);
  }
  if (!x2) {
    auto k = lj_general(t) ? k_adjoint<R, true> : k_adjoint<R, false>;
    DCM_LAUNCH(ctx, k, (unsigned)to.ntile, kBlock, 0, st, n, pos, rc, cell_start, a, A, (R)(0.5 * dlde), G, part,
               nwarp, bg, (const int32_t*)ctx->blk_max, order);
  }
  int r = check_launch(ctx, "lj_adjoint");
  if (r || !want) return r;
  int npair = nt * nt;
  for (int p = 0; p < npair; p += 4) {
    int q = std::min(4, npair - p);
    if ((r = reduce_partials(ctx, part + (int64_t)p * nwarp, nwarp, q, ctx->adj_pairs + p, false, st))) return r;
    if ((r = reduce_partials(ctx, part + (int64_t)(16 + p) * nwarp, nwarp, q, ctx->adj_pairs + 16 + p, false, st)))
      return r;
  }
  DCM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->adj_pairs + 32, ctx->p.eps, sizeof(double) * nt, cudaMemcpyHostToDevice, st));
  DCM_LAUNCH(ctx, k_mix_chain, 1, 1, 0, st, ctx->adj_pairs, ctx->adj_pairs + 16, nt, ctx->adj_pairs + 32, dparams);
  return check_launch(ctx, "lj_adjoint mix");
}

template int lj_adjoint<float>(dcm_ctx*, int64_t, const float4*, const float*, const int32_t*, const float4*, double,
                               float4*, double*, cudaStream_t);
template int lj_adjoint<double>(dcm_ctx*, int64_t, const dvec4*, const double*, const int32_t*, const dvec4*, double,
                                dvec4*, double*, cudaStream_t);

}  // namespace dcm
