// Verlet neighbour lists with a skin (Algorithm 2.2) and forces over them
// (Algorithm 2.3), used by dcm_step when params.skin > 0; with
// params.newton3 half lists whose pairs are evaluated once for both particles
// (the Newton's third law variant Section 4.2 points to).
//
// Build (at a rebuild): for every particle i, the j != i with
// |r_ij| < rc_i + skin, found by the same culled cell-row walk as the
// cell-list force kernel.  The lists of the 32 particles of a warp share one
// interleaved region (entry k of lane l at base + 32 k + l, base = 32 x the
// sum of the earlier warps' capacities) so that the force loop reads them
// coalesced.  Same-image neighbours are stored from the front of a lane's
// column as plain indices j; neighbours across the periodic boundary from the
// back as j | image code << 26, the code per dimension 0 = same image, 1 = j
// taken at x_j - L, 2 = i taken at x_i - L, so that every r_ij is formed
// with one rounding, exactly as in the cell walk.  The force loop therefore
// runs over plain entries without decoding and treats the few image entries
// apart.
//
// Between rebuilds particles are not rebinned and positions are not wrapped
// (the image codes stay valid); dcm_step rebuilds when the largest
// displacement since the build exceeds skin / 2 (then no pair can have moved
// from beyond rc_i + skin to within rc_i), and whenever the cutoffs are
// recomputed.
#include <algorithm>

#include "forces_core.cuh"

namespace dcm {

constexpr uint32_t kIdxBits = 26;
constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1;

// Walk the culled cell rows of particle i for radius rl and hand each row
// segment to the segment visitor v: v.plain(j0, j1, xi, yi, zi) for
// segments in i's own image (with i itself cut out) and v.image(j0, j1, xi,
// yi, zi, shx, shy, shz, code) for segments across the periodic boundary
// (xi.. the i coordinates and sh.. the j shifts of that image, code as stored
// in the lists).  The visitor tests r_ij^2 < rl^2 itself.
template <typename R, typename V>
__device__ __forceinline__ void walk_segments(const int32_t* __restrict__ start, const Grid<R>& g, int self,
                                              const typename RT<R>::R4& pi, R rl, V& v) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const R l = g.edge, il = g.inv_edge, ilx = g.inv_edge_x;
  const R rl2s = rl * rl * (R)1.000004;  // culling slack; the pair test is exact
  const int cx = cell_coord<R>(pi.x, g.edge_x, ilx, nx);
  const int cy = cell_coord<R>(pi.y, l, il, ny);
  const int cz = cell_coord<R>(pi.z, l, il, nz);
  const int H = (int)ceil(rl * il), Hx = (int)ceil(rl * ilx);
  for (int uz = cz - H; uz <= cz + H; ++uz) {
    R gz = uz > cz ? (R)uz * l - pi.z : (uz < cz ? pi.z - (R)(uz + 1) * l : (R)0);
    R gz2 = gz * gz;
    if (gz2 >= rl2s) continue;
    int wz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
    uint32_t zc = uz < 0 ? 1u : (uz >= nz ? 2u : 0u);
    R zi = zc == 2 ? pi.z - g.L[2] : pi.z;
    R zsh = zc == 1 ? -g.L[2] : (R)0;
    for (int uy = cy - H; uy <= cy + H; ++uy) {
      R gy = uy > cy ? (R)uy * l - pi.y : (uy < cy ? pi.y - (R)(uy + 1) * l : (R)0);
      R gyz2 = gz2 + gy * gy;
      if (gyz2 >= rl2s) continue;
      int wy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
      uint32_t yc = uy < 0 ? 1u : (uy >= ny ? 2u : 0u);
      R yi = yc == 2 ? pi.y - g.L[1] : pi.y;
      R ysh = yc == 1 ? -g.L[1] : (R)0;
      R wx = window_half_width(rl2s - gyz2);
      int ulo = max(ufloor<R>((pi.x - wx) * ilx - (R)5e-4), cx - Hx);
      int uhi = min(ufloor<R>((pi.x + wx) * ilx + (R)5e-4), cx + Hx);
      if (ulo > uhi) continue;  // a coordinate outside [0, L): no window
      const int64_t row = (int64_t)nx * (wy + (int64_t)ny * wz);
      const uint32_t yzc = (yc << 2) | (zc << 4);
      if (ulo < 0) {  // image -L in x: shift j
        int a1 = min(uhi, -1);
        int j0 = __ldg(start + row + ulo + nx), j1 = __ldg(start + row + a1 + nx + 1);
        v.image(j0, j1, pi.x, yi, zi, -g.L[0], ysh, zsh, yzc | 1u);
      }
      {
        int a0 = max(ulo, 0), a1 = min(uhi, nx - 1);
        if (a0 <= a1) {
          int j0 = __ldg(start + row + a0), j1 = __ldg(start + row + a1 + 1);
          if (yzc == 0) {
            v.plain(j0, min(j1, self), pi.x, yi, zi);
            v.plain(max(j0, self + 1), j1, pi.x, yi, zi);
          } else {
            v.image(j0, j1, pi.x, yi, zi, (R)0, ysh, zsh, yzc);
          }
        }
      }
      if (uhi >= nx) {  // image +L in x: shift i
        int a0 = max(ulo, nx);
        int j0 = __ldg(start + row + a0 - nx), j1 = __ldg(start + row + uhi - nx + 1);
        v.image(j0, j1, pi.x - g.L[0], yi, zi, (R)0, ysh, zsh, yzc | 2u);
      }
    }
  }
}

// Segment visitors of the build: counting, and filling a lane's column
// (plain entries from the front, image entries from the back, nothing
// written past the column's capacity).
// Which particle of a pair keeps it in a half list (Newton's third law form):
// the one with the larger cutoff, the lower index on a tie, so that its walk
// radius (its own cutoff plus the skin) covers the pair and every pair is
// kept exactly once.  Full lists (n3 = 0) keep every candidate.
template <typename R>
struct Owner {
  const R* __restrict__ rc;
  R rci, rc_max;
  int self, n3;
  __device__ __forceinline__ bool keeps(int j) const {
    if (!n3) return true;
    const R rcj = clamp_cutoff<R>(__ldg(rc + j), rc_max);
    return rci > rcj || (rci == rcj && self < j);
  }
};

template <typename R>
struct CountVisitor {
  const typename RT<R>::R4* __restrict__ pos;
  R rl2;
  int cnt;
  Owner<R> own;
  __device__ __forceinline__ void plain(int j0, int j1, R xi, R yi, R zi) {
    for (int j = j0; j < j1; ++j) {
      auto pj = ldg4(pos + j);
      R dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
      cnt += fma(dx, dx, fma(dy, dy, dz * dz)) < rl2 && own.keeps(j) ? 1 : 0;
    }
  }
  __device__ __forceinline__ void image(int j0, int j1, R xi, R yi, R zi, R shx, R shy, R shz, uint32_t) {
    for (int j = j0; j < j1; ++j) {
      auto pj = ldg4(pos + j);
      R dx = xi - (pj.x + shx), dy = yi - (pj.y + shy), dz = zi - (pj.z + shz);
      cnt += fma(dx, dx, fma(dy, dy, dz * dz)) < rl2 && own.keeps(j) ? 1 : 0;
    }
  }
};

// Predicated 32-bit store (no branch around it in the candidate loop).
__device__ __forceinline__ void store_if(bool p, uint32_t* addr, uint32_t v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.global.u32 [%0], %1;\n\t}" ::"l"(addr), "r"(v),
               "r"((uint32_t)p));  // no memory clobber: nothing in the build reads the lists back
}

template <typename R>
struct FillVisitor {
  const typename RT<R>::R4* __restrict__ pos;
  uint32_t* __restrict__ out;  // the lane's column: entry k at out[32 k]
  R rl2;
  int cap, kf, kb;
  Owner<R> own;
  __device__ __forceinline__ void plain(int j0, int j1, R xi, R yi, R zi) {
    const int lim = cap - kb;
    int k = kf;
    int j = j0;
    if constexpr (sizeof(R) == 4) {  // two candidates per packed r^2 (the same roundings as one at a time)
      // four position loads in flight: the walk does little arithmetic per
      // candidate, so without them it waits on the loads
      for (; j + 3 < j1; j += 4) {
        const float4 p0 = __ldg(pos + j), p1 = __ldg(pos + j + 1), p2 = __ldg(pos + j + 2), p3 = __ldg(pos + j + 3);
        const float2 dx = make_float2(xi - p0.x, xi - p1.x), dy = make_float2(yi - p0.y, yi - p1.y),
                     dz = make_float2(zi - p0.z, zi - p1.z);
        const float2 ex = make_float2(xi - p2.x, xi - p3.x), ey = make_float2(yi - p2.y, yi - p3.y),
                     ez = make_float2(zi - p2.z, zi - p3.z);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        const float2 s2 = __ffma2_rn(ex, ex, __ffma2_rn(ey, ey, __fmul2_rn(ez, ez)));
        const bool a0 = r2.x < rl2 && own.keeps(j), a1 = r2.y < rl2 && own.keeps(j + 1),
                   a2 = s2.x < rl2 && own.keeps(j + 2), a3 = s2.y < rl2 && own.keeps(j + 3);
        store_if(a0 && k < lim, out + (int64_t)k * 32, (uint32_t)j);
        k += a0 ? 1 : 0;
        store_if(a1 && k < lim, out + (int64_t)k * 32, (uint32_t)(j + 1));
        k += a1 ? 1 : 0;
        store_if(a2 && k < lim, out + (int64_t)k * 32, (uint32_t)(j + 2));
        k += a2 ? 1 : 0;
        store_if(a3 && k < lim, out + (int64_t)k * 32, (uint32_t)(j + 3));
        k += a3 ? 1 : 0;
      }
      for (; j + 1 < j1; j += 2) {
        const float4 p0 = __ldg(pos + j), p1 = __ldg(pos + j + 1);
        const float2 dx = make_float2(xi - p0.x, xi - p1.x), dy = make_float2(yi - p0.y, yi - p1.y),
                     dz = make_float2(zi - p0.z, zi - p1.z);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        const bool a0 = r2.x < rl2 && own.keeps(j), a1 = r2.y < rl2 && own.keeps(j + 1);
        store_if(a0 && k < lim, out + (int64_t)k * 32, (uint32_t)j);
        k += a0 ? 1 : 0;
        store_if(a1 && k < lim, out + (int64_t)k * 32, (uint32_t)(j + 1));
        k += a1 ? 1 : 0;
      }
    }
    for (; j < j1; ++j) {
      auto pj = ldg4(pos + j);
      R dx = xi - pj.x, dy = yi - pj.y, dz = zi - pj.z;
      const bool acc = fma(dx, dx, fma(dy, dy, dz * dz)) < rl2 && own.keeps(j);
      store_if(acc && k < lim, out + (int64_t)k * 32, (uint32_t)j);
      k += acc ? 1 : 0;
    }
    kf = k;
  }
  __device__ __forceinline__ void image(int j0, int j1, R xi, R yi, R zi, R shx, R shy, R shz, uint32_t code) {
    for (int j = j0; j < j1; ++j) {
      auto pj = ldg4(pos + j);
      R dx = xi - (pj.x + shx), dy = yi - (pj.y + shy), dz = zi - (pj.z + shz);
      if (fma(dx, dx, fma(dy, dy, dz * dz)) < rl2 && own.keeps(j)) {
        if (kf + kb < cap) out[(int64_t)(cap - 1 - kb) * 32] = (uint32_t)j | (code << kIdxBits);
        ++kb;
      }
    }
  }
};

template <typename R>
__device__ __forceinline__ R list_radius(R rc, R rc_max, R skin) {
  if (!(rc <= rc_max)) rc = rc_max;
  if (!(rc > (R)0)) rc = (R)0;
  return rc + skin;
}

template <typename R>
__global__ void __launch_bounds__(128) k_list_count(int64_t n, const typename RT<R>::R4* __restrict__ pos,
                                                    const R* __restrict__ rc, const int32_t* __restrict__ start,
                                                    Grid<R> g, R rc_max, R skin, int n3,
                                                    int32_t* __restrict__ capw) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = 0;
  if (i < n) {
    auto pi = ldg4(pos + i);
    R rl = list_radius<R>(rc[i], rc_max, skin);
    CountVisitor<R> v{pos, rl * rl, 0, Owner<R>{rc, clamp_cutoff<R>(rc[i], rc_max), rc_max, (int)i, n3}};
    walk_segments<R>(start, g, (int)i, pi, rl, v);
    cnt = v.cnt;
  }
  int m = cnt;
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) capw[i >> 5] = m;
}

// Fill lane columns of capacity capw[warp]: plain entries from the front,
// image entries from the back.  More than capw entries raise *flag (the lists
// are then incomplete and the caller counts exactly and fills again).
template <typename R>
__global__ void __maxnreg__(80) k_list_fill(int64_t n, const typename RT<R>::R4* __restrict__ pos,
                                                   const R* __restrict__ rc, const int32_t* __restrict__ start,
                                                   Grid<R> g, R rc_max, R skin, int n3,
                                                   const int32_t* __restrict__ capw,
                                                   const int32_t* __restrict__ offw, uint32_t* __restrict__ list,
                                                   int32_t* __restrict__ nnb, int32_t* __restrict__ nimg,
                                                   int32_t* __restrict__ flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto pi = ldg4(pos + i);
  R rl = list_radius<R>(rc[i], rc_max, skin);
  FillVisitor<R> v{pos, list + (int64_t)offw[i >> 5] * 32 + (threadIdx.x & 31), rl * rl, capw[i >> 5], 0, 0,
                   Owner<R>{rc, clamp_cutoff<R>(rc[i], rc_max), rc_max, (int)i, n3}};
  walk_segments<R>(start, g, (int)i, pi, rl, v);
  nnb[i] = v.kf;
  nimg[i] = v.kb;
  if (v.kf + v.kb > v.cap) atomicExch(flag, 1);
}

// Capacity bound of a list of radius R: the particles a sphere of radius R can
// hold at number density 1.3 (well above any liquid state of the workloads),
// plus a margin; a build that exceeds it is detected and redone exactly.
template <typename R>
__device__ __forceinline__ int list_cap_bound(R rl) {
  R v = (R)(4.18879020478639) * rl * rl * rl;  // 4/3 pi R^3
  return (int)(v * (R)1.3) + 24;
}

template <typename R>
__global__ void k_list_caps(int64_t n, const R* __restrict__ rc, R rc_max, R skin, int32_t* __restrict__ capw) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int cap = i < n ? list_cap_bound<R>(list_radius<R>(rc[i], rc_max, skin)) : 0;
  for (int o = 16; o > 0; o >>= 1) cap = max(cap, __shfl_xor_sync(0xffffffffu, cap, o));
  if ((threadIdx.x & 31) == 0) capw[i >> 5] = cap;
}

// Per-warp partials (E, W, pairs) as in the cell-list kernel.
template <typename R>
__device__ __forceinline__ void list_partials(R a, R b, int c, double* part, int64_t nslot) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    part[w] = (double)a;
    part[nslot + w] = (double)b;
    part[2 * nslot + w] = (double)c;
  }
}

// Pair term of the list kernels: accumulates j's contribution to i for the
// components (dx, dy, dz) of r_ij (rejected beyond rc_i).
template <typename R, bool TYPED>
__device__ __forceinline__ void list_pair(R dx, R dy, R dz, R rc2, int ti, R pjw, const ForceArgs<R>& a,
                                          const R* ushift, Acc<R>& c) {
  R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  bool acc = r2 < rc2;
  R inv = recip(r2);
  inv = acc ? inv : (R)0;
  if (TYPED) {
    int tj = type_of(pjw, a.ntypes);
    int tp = ti * a.ntypes + tj;
    R s2 = a.sig2[tp] * inv;
    R s6 = s2 * s2 * s2;
    R pv = a.eps24[tp] * s6 * fma((R)2, s6, (R)-1);
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
    R pv = s6 * fma((R)2, s6, (R)-1);
    R q = pv * inv;
    c.fx = fma(q, dx, c.fx);
    c.fy = fma(q, dy, c.fy);
    c.fz = fma(q, dz, c.fz);
    c.en += fma(s6, s6, -s6);
    c.vir += pv;
  }
  c.np += acc ? 1 : 0;
}

// r_ij of an image entry (code != 0), one rounding per component.
template <typename R>
__device__ __forceinline__ void image_delta(uint32_t code, const typename RT<R>::R4& pi,
                                            const typename RT<R>::R4& pj, const Grid<R>& g, R& dx, R& dy, R& dz) {
  uint32_t xc = code & 3, yc = (code >> 2) & 3, zc = code >> 4;
  dx = (xc == 2 ? pi.x - g.L[0] : pi.x) - (xc == 1 ? pj.x - g.L[0] : pj.x);
  dy = (yc == 2 ? pi.y - g.L[1] : pi.y) - (yc == 1 ? pj.y - g.L[1] : pj.y);
  dz = (zc == 2 ? pi.z - g.L[2] : pi.z) - (zc == 1 ? pj.z - g.L[2] : pj.z);
}

template <typename R, bool TYPED>
__device__ __forceinline__ void list_finish(const Acc<R>& c, const R* ushift, typename RT<R>::R4& out, R& e_out,
                                            R& w_out) {
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
}

// Forces over the lists (general form: any types, FP32 or FP64): the pair
// rule |r_ij| < rc_i is applied to every entry (the list holds the j within
// rc_i + skin at build time).
template <typename R, bool TYPED>
__global__ void __launch_bounds__(128) k_forces_list(int64_t n, const typename RT<R>::R4* __restrict__ pos,
                                                     const R* __restrict__ rc, const int32_t* __restrict__ nnb,
                                                     const int32_t* __restrict__ nimg,
                                                     const int32_t* __restrict__ capw,
                                                     const int32_t* __restrict__ offw,
                                                     const uint32_t* __restrict__ list, ForceArgs<R> a,
                                                     typename RT<R>::R4* __restrict__ force, double* __restrict__ part,
                                                     int64_t nwarp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  Acc<R> c;
  R e_out = 0, w_out = 0;
  if (i < n) {
    auto pi = ldg4(pos + i);
    R rci = rc[i];
    if (!(rci <= a.rc_max)) rci = a.rc_max;
    if (!(rci > (R)0)) rci = (R)0;
    const R rc2 = rci * rci;
    const int ti = TYPED ? type_of(pi.w, a.ntypes) : 0;
    R ushift[4] = {0, 0, 0, 0};
    if (a.shift && rc2 > (R)0) {
      for (int t = 0; t < (TYPED ? a.ntypes : 1); ++t) {
        int tp = ti * a.ntypes + t;
        R s2 = (TYPED ? a.sig2[tp] : (R)1) / rc2;
        R s6 = s2 * s2 * s2;
        ushift[t] = (TYPED ? a.eps4[tp] : (R)4) * s6 * (s6 - (R)1);
      }
    }
    const uint32_t* lp = list + (int64_t)offw[i >> 5] * 32 + (threadIdx.x & 31);
    const int m = nnb[i], cap = capw[i >> 5], mb = nimg[i];
#pragma unroll 2
    for (int k = 0; k < m; ++k) {
      int j = (int)__ldg(lp + (int64_t)k * 32);
      auto pj = ldg4(pos + j);
      list_pair<R, TYPED>(pi.x - pj.x, pi.y - pj.y, pi.z - pj.z, rc2, ti, pj.w, a, ushift, c);
    }
    for (int k = cap - mb; k < cap; ++k) {
      uint32_t e = __ldg(lp + (int64_t)k * 32);
      auto pj = ldg4(pos + (e & kIdxMask));
      R dx, dy, dz;
      image_delta<R>(e >> kIdxBits, pi, pj, a.g, dx, dy, dz);
      list_pair<R, TYPED>(dx, dy, dz, rc2, ti, pj.w, a, ushift, c);
    }
    typename RT<R>::R4 out;
    list_finish<R, TYPED>(c, ushift, out, e_out, w_out);
    force[i] = out;
  }
  if (part) list_partials<R>(e_out, w_out, c.np, part, nwarp);
}

// Forces over the lists, one type with eps = sigma = 1, FP32: the plain
// entries are taken two at a time with packed FP32x2 arithmetic (one
// instruction for both pairs wherever the operation allows), which halves the
// issue slots of the pair math.  With d = r_j - r_i (so that no packed operand
// needs negating), y = 1/r^2 (zero beyond rc_i) and s6 = y^3:
//   r.F/24 = s6 (2 s6 - 1),   -F_i/24 = sum (r.F/24) y d,   U/4 = s6 (s6 - 1).
// The reciprocal is refined exactly as in the cell kernel (one Newton step on
// the hardware approximation, the residual 1 - r^2 y0 formed by an FMA).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

struct PackedAcc {
  float2 fx, fy, fz, en, vir;
  int np;
};

// Two same-image neighbours p0, p1 of the particle at pi (cutoff^2 rc2).
__device__ __forceinline__ void packed_pair(const float4& pi, const float4& p0, const float4& p1, float rc2,
                                            PackedAcc& c) {
  const float2 two = f2(2.f, 2.f), m1 = f2(-1.f, -1.f);
  const float2 dx = f2(p0.x - pi.x, p1.x - pi.x);
  const float2 dy = f2(p0.y - pi.y, p1.y - pi.y);
  const float2 dz = f2(p0.z - pi.z, p1.z - pi.z);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  float y0, y1;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(r2.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(r2.y));
  const float2 e = f2(fmaf(-r2.x, y0, 1.f), fmaf(-r2.y, y1, 1.f));
  float2 y = f2(y0, y1);
  y = __ffma2_rn(y, e, y);
  const bool a0 = r2.x < rc2, a1 = r2.y < rc2;
  y = f2(a0 ? y.x : 0.f, a1 ? y.y : 0.f);
  const float2 s6 = __fmul2_rn(__fmul2_rn(y, y), y);
  const float2 pv = __fmul2_rn(s6, __ffma2_rn(s6, two, m1));  // r.F / 24
  const float2 q = __fmul2_rn(pv, y);
  c.fx = __ffma2_rn(q, dx, c.fx);
  c.fy = __ffma2_rn(q, dy, c.fy);
  c.fz = __ffma2_rn(q, dz, c.fz);
  c.en = __ffma2_rn(s6, __fadd2_rn(s6, m1), c.en);
  c.vir = __fadd2_rn(c.vir, pv);
  c.np += (int)a0 + (int)a1;
}

__global__ void __launch_bounds__(128) k_forces_list_x2(int64_t n, const float4* __restrict__ pos,
                                                        const float* __restrict__ rc, const int32_t* __restrict__ nnb,
                                                        const int32_t* __restrict__ nimg,
                                                        const int32_t* __restrict__ capw,
                                                        const int32_t* __restrict__ offw,
                                                        const uint32_t* __restrict__ list, ForceArgs<float> a,
                                                        float4* __restrict__ force, double* __restrict__ part,
                                                        int64_t nwarp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float e_out = 0.f, w_out = 0.f;
  int np = 0;
  if (i < n) {
    const float4 pi = __ldg(pos + i);
    float rci = __ldg(rc + i);
    if (!(rci <= a.rc_max)) rci = a.rc_max;
    if (!(rci > 0.f)) rci = 0.f;
    const float rc2 = rci * rci;
    const uint32_t* lp = list + (int64_t)offw[i >> 5] * 32 + (threadIdx.x & 31);
    const int m = nnb[i], cap = capw[i >> 5], mb = nimg[i];
    PackedAcc pc;
    pc.fx = pc.fy = pc.fz = pc.en = pc.vir = f2(0.f, 0.f);
    pc.np = 0;
    int k = 0;
    // four entries per iteration; the next four indices are requested before
    // this iteration's arithmetic (the list streams from DRAM once, so its
    // loads bypass L1 and leave it to the positions)
    if (k + 3 < m) {
      int e0 = (int)__ldcs(lp), e1 = (int)__ldcs(lp + 32), e2 = (int)__ldcs(lp + 64), e3 = (int)__ldcs(lp + 96);
      for (; k + 3 < m; k += 4) {
        const float4 p0 = __ldg(pos + e0), p1 = __ldg(pos + e1), p2 = __ldg(pos + e2), p3 = __ldg(pos + e3);
        if (k + 7 < m) {
          const uint32_t* q = lp + (int64_t)(k + 4) * 32;
          e0 = (int)__ldcs(q);
          e1 = (int)__ldcs(q + 32);
          e2 = (int)__ldcs(q + 64);
          e3 = (int)__ldcs(q + 96);
        }
        packed_pair(pi, p0, p1, rc2, pc);
        packed_pair(pi, p2, p3, rc2, pc);
      }
    }
    if (k + 1 < m) {
      const int j0 = (int)__ldg(lp + (int64_t)k * 32), j1 = (int)__ldg(lp + (int64_t)(k + 1) * 32);
      packed_pair(pi, __ldg(pos + j0), __ldg(pos + j1), rc2, pc);
      k += 2;
    }
    const float2 fx = pc.fx, fy = pc.fy, fz = pc.fz, en = pc.en, vir = pc.vir;
    np = pc.np;
    Acc<float> c;
    c.fx = -(fx.x + fx.y);
    c.fy = -(fy.x + fy.y);
    c.fz = -(fz.x + fz.y);
    c.en = en.x + en.y;
    c.vir = vir.x + vir.y;
    c.np = np;
    const float ushift0 = 0.f;
    if (k < m) {
      const int j = (int)__ldg(lp + (int64_t)k * 32);
      const float4 pj = __ldg(pos + j);
      list_pair<float, false>(pi.x - pj.x, pi.y - pj.y, pi.z - pj.z, rc2, 0, pj.w, a, &ushift0, c);
    }
    for (int kk = cap - mb; kk < cap; ++kk) {
      const uint32_t e = __ldg(lp + (int64_t)kk * 32);
      const float4 pj = __ldg(pos + (e & kIdxMask));
      float dx, dy, dz;
      image_delta<float>(e >> kIdxBits, pi, pj, a.g, dx, dy, dz);
      list_pair<float, false>(dx, dy, dz, rc2, 0, pj.w, a, &ushift0, c);
    }
    float ushift[4] = {0.f, 0.f, 0.f, 0.f};
    if (a.shift && rc2 > 0.f) {
      float s2 = 1.f / rc2, s6 = s2 * s2 * s2;
      ushift[0] = 4.f * s6 * (s6 - 1.f);
    }
    float4 out;
    list_finish<float, false>(c, ushift, out, e_out, w_out);
    force[i] = out;
    np = c.np;
  }
  if (part) list_partials<float>(e_out, w_out, np, part, nwarp);
}

// Half kick and drift without wrapping (the list's image codes stay valid),
// with the largest squared displacement since the build (as float bits; the
// values are non-negative, so integer max orders them).
template <typename R>
__global__ void k_kick_drift_nowrap(int64_t n, typename RT<R>::R4* __restrict__ pos, typename RT<R>::R4* __restrict__ vel,
                                    const typename RT<R>::R4* __restrict__ force,
                                    const typename RT<R>::R4* __restrict__ xb, R half_dt, R dt,
                                    int32_t* __restrict__ dmax, int kicks) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float d2 = 0.f;
  if (i < n) {
    auto p = pos[i];
    auto v = vel[i];
    auto f = force[i];
    for (int k = 0; k < kicks; ++k) {  // 2: also the previous step's second half kick
      v.x += half_dt * f.x;
      v.y += half_dt * f.y;
      v.z += half_dt * f.z;
    }
    p.x += dt * v.x;
    p.y += dt * v.y;
    p.z += dt * v.z;
    pos[i] = p;
    vel[i] = v;
    auto b = xb[i];
    R dx = p.x - b.x, dy = p.y - b.y, dz = p.z - b.z;
    d2 = (float)(dx * dx + dy * dy + dz * dz);
    if (!(d2 == d2)) d2 = 3.0e38f;  // NaN: force a rebuild
  }
  for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dmax, __float_as_int(d2));
}

// Wrap drifted positions into [0, L) and count cells (the rebuild's binning).
template <typename R>
__global__ void k_wrap_count(int64_t n, typename RT<R>::R4* __restrict__ pos, Grid<R> g, int32_t* __restrict__ cell,
                             int32_t* __restrict__ slot, int32_t* __restrict__ count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto p = pos[i];
  R* c3[3] = {&p.x, &p.y, &p.z};
  for (int d = 0; d < 3; ++d) {
    R x = *c3[d];
    R L = g.L[d];
    if (x >= L) x -= L;
    if (x < (R)0) {
      x += L;
      if (x >= L) x = (R)0;
    }
    *c3[d] = x;
  }
  pos[i] = p;
  int cx = cell_coord<R>(p.x, g.edge_x, g.inv_edge_x, g.n[0]);
  int cy = cell_coord<R>(p.y, g.edge, g.inv_edge, g.n[1]);
  int cz = cell_coord<R>(p.z, g.edge, g.inv_edge, g.n[2]);
  int c = cx + g.n[0] * (cy + g.n[1] * cz);
  cell[i] = c;
  slot[i] = atomicAdd(count + c, 1);
}

// Forces over half lists (Newton's third law form, params.newton3): every
// pair of a list is evaluated once, by its owner i (the particle with the
// larger cutoff; the lower index on a tie).  The pair term goes to i if
// |r_ij| < rc_i and, with the opposite sign, to j if |r_ij| < rc_j; each side
// takes half of U, minus its own U(rc) with the shifted energy.  So a pair
// within both cutoffs (the symmetric case) costs one evaluation for both
// particles, and a pair within one cutoff only (the asymmetric case of
// Section 2.4) goes to that particle alone, as in the i-centric rule.  The
// contributions to j (and i's own total, since other threads add to it) are
// added with atomics into the force array, which is cleared first; the
// order of those additions varies from run to run.
// Atomic add of (x, y, z, w) to a force record: one 16-byte vector atomic in
// FP32 (sm_90 and later), four scalar ones in FP64.
template <typename R>
__device__ __forceinline__ void add_force4(typename RT<R>::R4* f, R x, R y, R z, R w) {
  if constexpr (sizeof(R) == 4) {
    atomicAdd(f, make_float4(x, y, z, w));
  } else {
    atomicAdd(&f->x, x);
    atomicAdd(&f->y, y);
    atomicAdd(&f->z, z);
    atomicAdd(&f->w, w);
  }
}

template <typename R, bool TYPED>
__global__ void __launch_bounds__(128) k_forces_list_n3(int64_t n, const typename RT<R>::R4* __restrict__ pos,
                                                        const R* __restrict__ rc, const int32_t* __restrict__ nnb,
                                                        const int32_t* __restrict__ nimg,
                                                        const int32_t* __restrict__ capw,
                                                        const int32_t* __restrict__ offw,
                                                        const uint32_t* __restrict__ list, ForceArgs<R> a,
                                                        typename RT<R>::R4* __restrict__ force,
                                                        double* __restrict__ part, int64_t nwarp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double E = 0.0, W = 0.0;
  int np = 0;
  if (i < n) {
    const auto pi = ldg4(pos + i);
    const R rci = clamp_cutoff<R>(rc[i], a.rc_max);
    const R rc2 = rci * rci;
    const int ti = TYPED ? type_of(pi.w, a.ntypes) : 0;
    // U(rc) per pair type: of i's cutoff (for i's half) and of j's (for j's)
    auto ushift = [&](int tp, R r2c) -> R {
      if (!a.shift || !(r2c > (R)0)) return (R)0;
      const R s2 = a.sig2[tp] / r2c, s6 = s2 * s2 * s2;
      return a.eps4[tp] * s6 * (s6 - (R)1);
    };
    R fx = 0, fy = 0, fz = 0, ei = 0;
    const uint32_t* lp = list + (int64_t)offw[i >> 5] * 32 + (threadIdx.x & 31);
    const int m = nnb[i], cap = capw[i >> 5], mb = nimg[i];
    auto pair = [&](uint32_t e, bool image) {
      const int j = (int)(e & kIdxMask);
      const auto pj = ldg4(pos + j);
      R dx, dy, dz;
      if (image)
        image_delta<R>(e >> kIdxBits, pi, pj, a.g, dx, dy, dz);
      else {
        dx = pi.x - pj.x;
        dy = pi.y - pj.y;
        dz = pi.z - pj.z;
      }
      const R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
      const R rcj = clamp_cutoff<R>(__ldg(rc + j), a.rc_max);
      const bool acc_i = r2 < rc2, acc_j = r2 < rcj * rcj;
      if (!acc_i && !acc_j) return;
      const int tj = TYPED ? type_of(pj.w, a.ntypes) : 0;
      const int tp = ti * a.ntypes + tj;
      const R inv = recip(r2);
      const R s2 = a.sig2[tp] * inv;
      const R s6 = s2 * s2 * s2;
      const R pv = a.eps24[tp] * s6 * fma((R)2, s6, (R)-1);  // r . F_ij
      const R fs = pv * inv;
      const R u = a.eps4[tp] * s6 * (s6 - (R)1);
      if (acc_i) {
        fx = fma(fs, dx, fx);
        fy = fma(fs, dy, fy);
        fz = fma(fs, dz, fz);
        ei += u - ushift(tp, rc2);
        W += 0.5 * (double)pv;
        ++np;
      }
      if (acc_j) {
        const R ej = (R)0.5 * (u - ushift(tp, rcj * rcj));
        add_force4<R>(force + j, -fs * dx, -fs * dy, -fs * dz, ej);
        E += (double)ej;
        W += 0.5 * (double)pv;
        ++np;
      }
    };
    for (int k = 0; k < m; ++k) pair(__ldg(lp + (int64_t)k * 32), false);
    for (int k = cap - mb; k < cap; ++k) pair(__ldg(lp + (int64_t)k * 32), true);
    ei *= (R)0.5;
    E += (double)ei;
    add_force4<R>(force + i, fx, fy, fz, ei);
  }
  if (part) {
    for (int o = 16; o > 0; o >>= 1) {
      E += __shfl_xor_sync(0xffffffffu, E, o);
      W += __shfl_xor_sync(0xffffffffu, W, o);
      np += __shfl_xor_sync(0xffffffffu, np, o);
    }
    if ((threadIdx.x & 31) == 0) {
      const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
      part[w] = E;
      part[nwarp + w] = W;
      part[2 * nwarp + w] = (double)np;
    }
  }
}

// The half-list kernel for one type with eps = sigma = 1 in FP32: two plain
// entries per step with packed FP32x2 arithmetic for the pair terms they
// share (with d = r_i - r_j, y = 1/r^2, s6 = y^3: r.F = 24 s6 (2 s6 - 1),
// F_ij = (r.F) y d, U = 4 s6 (s6 - 1)), then each side masked by its own
// cutoff: i's sums take the slots with r^2 < rc_i^2, and j's vector atomic is
// issued for the slots with r^2 < rc_j^2.  No branch skips a slot that
// neither cutoff reaches (its terms are masked out).  Odd and image entries
// take the scalar step of k_forces_list_n3; per-thread energy and virial sums
// in FP32, as in the full-list kernels.
__global__ void __launch_bounds__(128) k_forces_list_n3_x2(int64_t n, const float4* __restrict__ pos,
                                                           const float* __restrict__ rc,
                                                           const int32_t* __restrict__ nnb,
                                                           const int32_t* __restrict__ nimg,
                                                           const int32_t* __restrict__ capw,
                                                           const int32_t* __restrict__ offw,
                                                           const uint32_t* __restrict__ list, ForceArgs<float> a,
                                                           float4* __restrict__ force, double* __restrict__ part,
                                                           int64_t nwarp) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float ei = 0.f, ej = 0.f, w = 0.f;
  int np = 0;
  if (i < n) {
    const float4 pi = __ldg(pos + i);
    const float rci = clamp_cutoff<float>(__ldg(rc + i), a.rc_max), rc2 = rci * rci;
    // U(rc) of a cutoff for the shifted energy (zero without the shift)
    auto ushift = [&](float r2c) -> float {
      if (!a.shift || !(r2c > 0.f)) return 0.f;
      const float s2 = 1.f / r2c, s6 = s2 * s2 * s2;
      return 4.f * s6 * (s6 - 1.f);
    };
    const float usi = ushift(rc2);
    const uint32_t* lp = list + (int64_t)offw[i >> 5] * 32 + (threadIdx.x & 31);
    const int m = nnb[i], cap = capw[i >> 5], mb = nimg[i];
    float2 fx = f2(0.f, 0.f), fy = f2(0.f, 0.f), fz = f2(0.f, 0.f);
    const float2 two = f2(2.f, 2.f), m1 = f2(-1.f, -1.f);
    int k = 0;
    for (; k + 1 < m; k += 2) {
      const int j0 = (int)__ldcs(lp + (int64_t)k * 32), j1 = (int)__ldcs(lp + (int64_t)(k + 1) * 32);
      const float4 p0 = __ldg(pos + j0), p1 = __ldg(pos + j1);
      const float rj0 = clamp_cutoff<float>(__ldg(rc + j0), a.rc_max), rj1 = clamp_cutoff<float>(__ldg(rc + j1), a.rc_max);
      const float2 dx = f2(pi.x - p0.x, pi.x - p1.x), dy = f2(pi.y - p0.y, pi.y - p1.y), dz = f2(pi.z - p0.z, pi.z - p1.z);
      const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
      float y0, y1;
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(r2.x));
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y1) : "f"(r2.y));
      float2 y = f2(y0, y1);
      y = __ffma2_rn(y, f2(fmaf(-r2.x, y0, 1.f), fmaf(-r2.y, y1, 1.f)), y);
      const bool ai0 = r2.x < rc2, ai1 = r2.y < rc2;
      const bool aj0 = r2.x < rj0 * rj0, aj1 = r2.y < rj1 * rj1;
      y = f2(ai0 || aj0 ? y.x : 0.f, ai1 || aj1 ? y.y : 0.f);
      const float2 s6 = __fmul2_rn(__fmul2_rn(y, y), y);
      const float2 pv = __fmul2_rn(f2(24.f, 24.f), __fmul2_rn(s6, __ffma2_rn(s6, two, m1)));  // r . F_ij
      const float2 fs = __fmul2_rn(pv, y);
      const float2 u = __fmul2_rn(f2(4.f, 4.f), __fmul2_rn(s6, __fadd2_rn(s6, m1)));
      const float2 fi = f2(ai0 ? fs.x : 0.f, ai1 ? fs.y : 0.f);
      fx = __ffma2_rn(fi, dx, fx);
      fy = __ffma2_rn(fi, dy, fy);
      fz = __ffma2_rn(fi, dz, fz);
      ei += (ai0 ? u.x - usi : 0.f) + (ai1 ? u.y - usi : 0.f);
      w += (ai0 ? 0.5f * pv.x : 0.f) + (ai1 ? 0.5f * pv.y : 0.f);
      np += (int)ai0 + (int)ai1;
      if (aj0) {
        const float e0 = 0.5f * (u.x - ushift(rj0 * rj0));
        add_force4<float>(force + j0, -fs.x * dx.x, -fs.x * dy.x, -fs.x * dz.x, e0);
        ej += e0;
        w += 0.5f * pv.x;
        ++np;
      }
      if (aj1) {
        const float e1 = 0.5f * (u.y - ushift(rj1 * rj1));
        add_force4<float>(force + j1, -fs.y * dx.y, -fs.y * dy.y, -fs.y * dz.y, e1);
        ej += e1;
        w += 0.5f * pv.y;
        ++np;
      }
    }
    // the odd entry and the image entries: the scalar step
    float sfx = 0.f, sfy = 0.f, sfz = 0.f, sei = 0.f;
    auto pair = [&](uint32_t e, bool image) {
      const int j = (int)(e & kIdxMask);
      const float4 pj = __ldg(pos + j);
      float dx, dy, dz;
      if (image)
        image_delta<float>(e >> kIdxBits, pi, pj, a.g, dx, dy, dz);
      else {
        dx = pi.x - pj.x;
        dy = pi.y - pj.y;
        dz = pi.z - pj.z;
      }
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const float rcj = clamp_cutoff<float>(__ldg(rc + j), a.rc_max);
      const bool acc_i = r2 < rc2, acc_j = r2 < rcj * rcj;
      if (!acc_i && !acc_j) return;
      const float inv = recip(r2);
      const float s6 = inv * inv * inv;
      const float pv = 24.f * s6 * fmaf(2.f, s6, -1.f);
      const float fs = pv * inv;
      const float u = 4.f * s6 * (s6 - 1.f);
      if (acc_i) {
        sfx = fmaf(fs, dx, sfx);
        sfy = fmaf(fs, dy, sfy);
        sfz = fmaf(fs, dz, sfz);
        sei += u - usi;
        w += 0.5f * pv;
        ++np;
      }
      if (acc_j) {
        const float e1 = 0.5f * (u - ushift(rcj * rcj));
        add_force4<float>(force + j, -fs * dx, -fs * dy, -fs * dz, e1);
        ej += e1;
        w += 0.5f * pv;
        ++np;
      }
    };
    if (k < m) pair(__ldg(lp + (int64_t)k * 32), false);
    for (int kk = cap - mb; kk < cap; ++kk) pair(__ldg(lp + (int64_t)kk * 32), true);
    ei = 0.5f * (ei + sei);
    add_force4<float>(force + i, (fx.x + fx.y) + sfx, (fy.x + fy.y) + sfy, (fz.x + fz.y) + sfz, ei);
  }
  if (part) {
    double E = (double)ei + (double)ej, W = (double)w;
    for (int o = 16; o > 0; o >>= 1) {
      E += __shfl_xor_sync(0xffffffffu, E, o);
      W += __shfl_xor_sync(0xffffffffu, W, o);
      np += __shfl_xor_sync(0xffffffffu, np, o);
    }
    if ((threadIdx.x & 31) == 0) {
      const int64_t wi = i >> 5;
      part[wi] = E;
      part[nwarp + wi] = W;
      part[2 * nwarp + wi] = (double)np;
    }
  }
}

// ---- launchers -------------------------------------------------------------------

static int ensure_list_capacity(dcm_ctx* ctx, int64_t need) {
  if (need <= ctx->list_cap) return DCM_OK;
  if (ctx->list) cudaFree(ctx->list);
  ctx->list = nullptr;
  ctx->list_cap = 0;
  int64_t cap = need + need / 8 + 1024;
  if (cudaMalloc((void**)&ctx->list, sizeof(uint32_t) * cap) != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, DCM_ERR_NOMEM, "neighbour lists need %lld entries", (long long)need);
  }
  ctx->list_cap = cap;
  return DCM_OK;
}

// Build: bounded capacities -> one walk; on overflow, exact count + fill.
template <typename R>
int list_build(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc, cudaStream_t st) {
  Grid<R> g = cell_grid<R>(ctx);
  R skin = (R)ctx->p.skin, rcm = (R)ctx->p.rc_max;
  const int n3 = ctx->p.newton3;
  int64_t nblk = (n + 127) / 128, nw = nblk * 4;
  stage_begin(ctx, DCM_STAGE_LISTS, st);
  if (n > 0) DCM_LAUNCH(ctx, k_list_caps<R>, (unsigned)nblk, 128, 0, st, n, rc, rcm, skin, ctx->capw);
  int r = exclusive_scan(ctx, ctx->capw, ctx->offw, nw, st);
  if (r) return r;
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->lflag, 0, sizeof(int32_t), st));
  DCM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->host_status + 1, ctx->offw + nw, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DCM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if ((r = ensure_list_capacity(ctx, (int64_t)ctx->host_status[1] * 32))) return r;
  if (n > 0)
    DCM_LAUNCH(ctx, k_list_fill<R>, (unsigned)nblk, 128, 0, st, n, pos, rc, ctx->cell_start, g, rcm, skin, n3,
               ctx->capw, ctx->offw, ctx->list, ctx->nnb, ctx->nimg, ctx->lflag);
  DCM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->host_status + 3, ctx->lflag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DCM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (ctx->host_status[3]) {
    // some list outgrew its bound: count exactly, then fill again
    if (n > 0)
      DCM_LAUNCH(ctx, k_list_count<R>, (unsigned)nblk, 128, 0, st, n, pos, rc, ctx->cell_start, g, rcm, skin, n3,
                 ctx->capw);
    if ((r = exclusive_scan(ctx, ctx->capw, ctx->offw, nw, st))) return r;
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->lflag, 0, sizeof(int32_t), st));
    DCM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->host_status + 1, ctx->offw + nw, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DCM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if ((r = ensure_list_capacity(ctx, (int64_t)ctx->host_status[1] * 32))) return r;
    if (n > 0)
      DCM_LAUNCH(ctx, k_list_fill<R>, (unsigned)nblk, 128, 0, st, n, pos, rc, ctx->cell_start, g, rcm, skin, n3,
                 ctx->capw, ctx->offw, ctx->list, ctx->nnb, ctx->nimg, ctx->lflag);
  }
  DCM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->xbuild, pos, sizeof(typename RT<R>::R4) * n, cudaMemcpyDeviceToDevice, st));
  stage_end(ctx, DCM_STAGE_LISTS, st);
  ctx->list_valid = 1;
  return check_launch(ctx, "list_build");
}

// The list kernels sum energy and virial whether or not the caller reads
// them: a force-only instance of the packed kernel (40 registers against 48)
// ran 3% slower, its higher occupancy costing this L1-bound loop hits.
template <typename R>
int list_forces(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc, typename RT<R>::R4* force,
                double* totals, cudaStream_t st, bool energies) {
  (void)energies;
  if (n <= 0) {
    if (totals) DCM_CUDA_TRY(ctx, cudaMemsetAsync(totals, 0, 3 * sizeof(double), st));
    return DCM_OK;
  }
  ForceArgs<R> a;
  a.g = cell_grid<R>(ctx);
  LJTable t = lj_table(ctx->p);
  a.ntypes = t.ntypes;
  for (int k = 0; k < 16; ++k) {
    a.eps24[k] = (R)t.deps24[k];
    a.eps4[k] = (R)t.deps4[k];
    a.sig2[k] = (R)t.dsig2[k];
  }
  a.shift = ctx->p.shift_energy;
  a.rc_max = (R)ctx->p.rc_max;
  int64_t nblk = (n + 127) / 128, nwarp = nblk * 4;
  if (totals && nwarp > ctx->red_cap) return set_error(ctx, DCM_ERR_CAPACITY, "force reduction too large");
  double* part = totals ? ctx->red : nullptr;
  auto kern = lj_general(t) ? k_forces_list<R, true> : k_forces_list<R, false>;
  stage_begin(ctx, DCM_STAGE_FORCES, st);
  if (ctx->p.newton3) {
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(force, 0, sizeof(typename RT<R>::R4) * n, st));
    bool packed3 = false;
    if constexpr (sizeof(R) == 4) {
      if (!lj_general(t)) {
        DCM_LAUNCH(ctx, k_forces_list_n3_x2, (unsigned)nblk, 128, 0, st, n, pos, rc, ctx->nnb, ctx->nimg, ctx->capw,
                   ctx->offw, ctx->list, a, force, part, nwarp);
        packed3 = true;
      }
    }
    if (!packed3) {
      auto k3 = lj_general(t) ? k_forces_list_n3<R, true> : k_forces_list_n3<R, false>;
      DCM_LAUNCH(ctx, k3, (unsigned)nblk, 128, 0, st, n, pos, rc, ctx->nnb, ctx->nimg, ctx->capw, ctx->offw,
                 ctx->list, a, force, part, nwarp);
    }
    stage_end(ctx, DCM_STAGE_FORCES, st);
    int r = check_launch(ctx, "list_forces");
    if (r) return r;
    if (totals) return reduce_partials(ctx, part, nwarp, 3, totals, false, st);
    return DCM_OK;
  }
  bool packed = false;
  if constexpr (sizeof(R) == 4) {
    if (!lj_general(t)) {
      DCM_LAUNCH(ctx, k_forces_list_x2, (unsigned)nblk, 128, 0, st, n, pos, rc, ctx->nnb, ctx->nimg, ctx->capw,
                 ctx->offw, ctx->list, a, force, part, nwarp);
      packed = true;
    }
  }
  if (!packed)
    DCM_LAUNCH(ctx, kern, (unsigned)nblk, 128, 0, st, n, pos, rc, ctx->nnb, ctx->nimg, ctx->capw, ctx->offw,
               ctx->list, a, force, part, nwarp);
  stage_end(ctx, DCM_STAGE_FORCES, st);
  int r = check_launch(ctx, "list_forces");
  if (r) return r;
  if (totals) return reduce_partials(ctx, part, nwarp, 3, totals, false, st);
  return DCM_OK;
}

// Half kick + drift (no wrap); returns through *rebuild whether the largest
// displacement since the build exceeds skin / 2 (synchronous read).
template <typename R>
int list_kick_drift(dcm_ctx* ctx, dcm_state* s, int64_t n, R hdt, R dt, int kicks, bool* rebuild, cudaStream_t st) {
  using R4 = typename RT<R>::R4;
  int c = s->cur;
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dmax, 0, sizeof(int32_t), st));
  if (n > 0)
    DCM_LAUNCH(ctx, k_kick_drift_nowrap<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, (R4*)s->pos[c],
               (R4*)s->vel[c], (const R4*)s->force, (const R4*)ctx->xbuild, hdt, dt, ctx->dmax, kicks);
  DCM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->host_status + 2, ctx->dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DCM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  int bits = ctx->host_status[2];
  float d2;
  memcpy(&d2, &bits, sizeof(d2));
  double half = 0.5 * ctx->p.skin;
  *rebuild = !((double)d2 <= half * half);
  return check_launch(ctx, "list_kick_drift");
}

template <typename R>
int list_wrap_count(dcm_ctx* ctx, dcm_state* s, int64_t n, cudaStream_t st) {
  using R4 = typename RT<R>::R4;
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cell_count, 0, sizeof(int32_t) * ctx->ncell, st));
  if (n > 0)
    DCM_LAUNCH(ctx, k_wrap_count<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, (R4*)s->pos[s->cur],
               cell_grid<R>(ctx), ctx->cell, ctx->slot, ctx->cell_count);
  return check_launch(ctx, "list_wrap_count");
}

template int list_build<float>(dcm_ctx*, int64_t, const float4*, const float*, cudaStream_t);
template int list_build<double>(dcm_ctx*, int64_t, const dvec4*, const double*, cudaStream_t);
template int list_forces<float>(dcm_ctx*, int64_t, const float4*, const float*, float4*, double*, cudaStream_t,
                                bool);
template int list_forces<double>(dcm_ctx*, int64_t, const dvec4*, const double*, dvec4*, double*, cudaStream_t,
                                 bool);
template int list_kick_drift<float>(dcm_ctx*, dcm_state*, int64_t, float, float, int, bool*, cudaStream_t);
template int list_kick_drift<double>(dcm_ctx*, dcm_state*, int64_t, double, double, int, bool*, cudaStream_t);
template int list_wrap_count<float>(dcm_ctx*, dcm_state*, int64_t, cudaStream_t);
template int list_wrap_count<double>(dcm_ctx*, dcm_state*, int64_t, cudaStream_t);

}  // namespace dcm
