// Lennard-Jones forces with per-particle cutoffs (Section 2.4, Algorithms 2.2
// and 2.3): i-centric, no Newton's third law, over cell lists.
//
// One thread per particle i in cell-sorted order (a warp therefore covers a
// few neighbouring cells and walks nearly the same neighbour rows).  The
// stencil is culled per particle (Section 2.3's small-bin idea taken to the
// particle level): a row of cells (fixed y, z offset) is visited only if its
// y-z slab lies within rc_i, and only the x-range of cells the sphere of
// radius rc_i actually reaches.  Cells along x are contiguous in the sorted
// order, so every row segment is one contiguous run of j particles.
//
// Periodic images are formed without rounding: an image shifted by -L is
// taken as x_j - L (exact, x_j >= L/2 whenever the pair can be accepted) and
// one shifted by +L as x_i - L on the i side (exact for the same reason), so
// each component r_ij carries a single rounding in FP32.
//
// Pair arithmetic is branch-free: rejected candidates get 1/r^2 = 0, which
// zeroes every term.
#include <algorithm>
#include <climits>
#include <cmath>

#include "forces_core.cuh"

namespace dcm {

// Per-warp partial sums of (E, W, pairs): summed across the warp in the
// working precision (32 terms), then stored as one FP64 partial per warp;
// no block barrier, so warps that finish early do not wait.
template <typename R>
__device__ __forceinline__ void warp_partials3(R a, R b, int c, double* part, int64_t nslot) {
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

template <typename R, bool TYPED>
__global__ void __launch_bounds__(kForceBlock) k_forces(int64_t n, const typename RT<R>::R4* __restrict__ pos,
                                                        const R* __restrict__ rc, const int32_t* __restrict__ start,
                                                        ForceArgs<R> a, typename RT<R>::R4* __restrict__ force,
                                                        double* __restrict__ part, int64_t nwarp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  R e_out = 0, w_out = 0;
  int np = 0;
  if (i < n) force[i] = force_one<R, TYPED>(pos, start, a.g, a, (int)i, ldg4(pos + i), rc[i], e_out, w_out, np);
  if (part) warp_partials3<R>(e_out, w_out, np, part, nwarp);
}

// The same walk with the packed two-candidates-per-instruction pair loop
// (one type, FP32, eps = sigma = 1).  Blocks of two warps: a block retires
// only when its slowest warp is done, and the row windows of neighbouring
// particles differ, so small blocks keep the SMs fuller (measured: 64
// threads 0.4% faster than 128, 32 threads 3% and 1024 threads 14% slower).
constexpr int kX2Block = 64;
__global__ void __launch_bounds__(kX2Block, 16) k_forces_x2(int64_t n, const float4* __restrict__ pos,
                                                           const float* __restrict__ rc,
                                                           const int32_t* __restrict__ start, ForceArgs<float> a,
                                                           float4* __restrict__ force, double* __restrict__ part,
                                                           int64_t nwarp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float e_out = 0, w_out = 0;
  int np = 0;
  if (i < n) force[i] = force_one<float, false, true>(pos, start, a.g, a, (int)i, __ldg(pos + i), rc[i], e_out, w_out, np);
  if (part) warp_partials3<float>(e_out, w_out, np, part, nwarp);
}

// The packed walk for one or two types with per-type eps and sigma (FP32).
__global__ void __launch_bounds__(kX2Block, 16) k_forces_x2t(int64_t n, const float4* __restrict__ pos,
                                                             const float* __restrict__ rc,
                                                             const int32_t* __restrict__ start, ForceArgs<float> a,
                                                             float4* __restrict__ force, double* __restrict__ part,
                                                             int64_t nwarp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float e_out = 0, w_out = 0;
  int np = 0;
  if (i < n) force[i] = force_one<float, true, true>(pos, start, a.g, a, (int)i, __ldg(pos + i), rc[i], e_out, w_out, np);
  if (part) warp_partials3<float>(e_out, w_out, np, part, nwarp);
}

// ----------------------------------------------------------------------------
// Tile kernel (one type, FP32): the warp's 32 particles share one x-line of
// cells, so for every row offset (dy, dz) their windows lie in one grid row;
// the warp stages the union of the windows (and the cell starts around it)
// in shared memory with coalesced loads, then every lane runs the packed pair
// loop of its own window from the tile.  Warps whose particles span two
// x-lines, or whose stencil reaches a periodic boundary or a tile overflows,
// take the cell-row walk of k_forces_x2.
// ----------------------------------------------------------------------------
constexpr int kTileWarps = 4;
constexpr int kTileCap = 128;   // staged particles per warp and row
constexpr int kTileCells = 40;  // staged cell starts per warp and row

__global__ void __launch_bounds__(32 * kTileWarps) k_forces_tile(int64_t n, const float4* __restrict__ pos,
                                                                 const float* __restrict__ rc,
                                                                 const int32_t* __restrict__ start,
                                                                 ForceArgs<float> a, float4* __restrict__ force,
                                                                 double* __restrict__ part, int64_t nwarp) {
  __shared__ float4 tile[kTileWarps][kTileCap];
  __shared__ int32_t cst[kTileWarps][kTileCells];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  const Grid<float>& g = a.g;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const float l = g.edge, il = g.inv_edge, ilx = g.inv_edge_x;
  const float4 pi = valid ? __ldg(pos + i) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float rc_in = valid ? __ldg(rc + i) : 0.f;
  float rci = rc_in;
  if (!(rci <= a.rc_max)) rci = a.rc_max;
  if (!(rci > 0.f)) rci = 0.f;
  const int cx = cell_coord<float>(pi.x, g.edge_x, ilx, nx), cy = cell_coord<float>(pi.y, l, il, ny),
            cz = cell_coord<float>(pi.z, l, il, nz);
  const int H = (int)ceilf(rci * il), Hx = (int)ceilf(rci * ilx);
  int Hm = H, Hxm = Hx, cmin = cx, cmax = cx;
  for (int o = 16; o > 0; o >>= 1) {
    Hm = max(Hm, __shfl_xor_sync(FULL, Hm, o));
    Hxm = max(Hxm, __shfl_xor_sync(FULL, Hxm, o));
    cmin = min(cmin, __shfl_xor_sync(FULL, cmin, o));
    cmax = max(cmax, __shfl_xor_sync(FULL, cmax, o));
  }
  const int cy0 = __shfl_sync(FULL, cy, 0), cz0 = __shfl_sync(FULL, cz, 0);
  const bool tiled = __all_sync(FULL, valid && cy == cy0 && cz == cz0) && cmin - Hxm >= 0 && cmax + Hxm < nx &&
                     cy0 - Hm >= 0 && cy0 + Hm < ny && cz0 - Hm >= 0 && cz0 + Hm < nz &&
                     (cmax - cmin) + 2 * Hxm + 2 <= kTileCells;
  float e_out = 0.f, w_out = 0.f;
  int np = 0;
  if (!tiled) {
    if (valid) force[i] = force_one<float, false, true>(pos, start, g, a, (int)i, pi, rc_in, e_out, w_out, np);
  } else {
    Acc2 c2;
    const float rc2 = rci * rci, rc2s = rc2 * 1.000004f;
    const int self = (int)i;
    for (int dz = -Hm; dz <= Hm; ++dz) {
      const int uz = cz0 + dz;
      const float gz = uz > cz ? (float)uz * l - pi.z : (uz < cz ? pi.z - (float)(uz + 1) * l : 0.f);
      for (int dy = -Hm; dy <= Hm; ++dy) {
        const int uy = cy0 + dy;
        const float gy = uy > cy ? (float)uy * l - pi.y : (uy < cy ? pi.y - (float)(uy + 1) * l : 0.f);
        const float gyz2 = gz * gz + gy * gy;
        bool has = dz >= -H && dz <= H && dy >= -H && dy <= H && gyz2 < rc2s;
        int ulo = 0, uhi = -1;
        if (has) {
          const float wx = window_half_width(rc2s - gyz2);
          ulo = max(ufloor<float>((pi.x - wx) * ilx - 5e-4f), cx - Hx);
          uhi = min(ufloor<float>((pi.x + wx) * ilx + 5e-4f), cx + Hx);
          has = ulo <= uhi;
        }
        if (__ballot_sync(FULL, has) == 0) continue;
        int umin = has ? ulo : INT_MAX, umax = has ? uhi : INT_MIN;
        for (int o = 16; o > 0; o >>= 1) {
          umin = min(umin, __shfl_xor_sync(FULL, umin, o));
          umax = max(umax, __shfl_xor_sync(FULL, umax, o));
        }
        const int64_t row = (int64_t)nx * (uy + (int64_t)ny * uz);
        const int ncs = umax - umin + 2;  // <= kTileCells: the stencil spans at most that many cells
        __syncwarp();                     // the previous row's tile is no longer read
        for (int k = lane; k < ncs; k += 32) cst[wid][k] = __ldg(start + row + umin + k);
        __syncwarp();
        const int base = cst[wid][0], cnt = cst[wid][ncs - 1] - base;
        const int j0 = has ? cst[wid][ulo - umin] : 0, j1 = has ? cst[wid][uhi - umin + 1] : 0;
        const bool centre = dz == 0 && dy == 0;
        if (cnt <= kTileCap) {
          for (int k = lane; k < cnt; k += 32) tile[wid][k] = __ldg(pos + base + k);
          __syncwarp();
          if (has) {
            const float4* tp = tile[wid] - base;  // indexed by the global slot j
            if (centre) {
              pair_range_x2<false, true>(tp, j0, self, pi.x, pi.y, pi.z, 0.f, 0.f, 0.f, rc2, c2);
              pair_range_x2<false, true>(tp, self + 1, j1, pi.x, pi.y, pi.z, 0.f, 0.f, 0.f, rc2, c2);
            } else {
              pair_range_x2<false, true>(tp, j0, j1, pi.x, pi.y, pi.z, 0.f, 0.f, 0.f, rc2, c2);
            }
          }
        } else if (has) {  // too many to stage: read this row from global memory
          if (centre) {
            pair_range_x2<false>(pos, j0, self, pi.x, pi.y, pi.z, 0.f, 0.f, 0.f, rc2, c2);
            pair_range_x2<false>(pos, self + 1, j1, pi.x, pi.y, pi.z, 0.f, 0.f, 0.f, rc2, c2);
          } else {
            pair_range_x2<false>(pos, j0, j1, pi.x, pi.y, pi.z, 0.f, 0.f, 0.f, rc2, c2);
          }
        }
      }
    }
    float ush = 0.f;
    if (a.shift && rc2 > 0.f) {
      const float s2 = 1.f / rc2, s6 = s2 * s2 * s2;
      ush = 4.f * s6 * (s6 - 1.f);
    }
    const float en = c2.en.x + c2.en.y;
    np = c2.np;
    e_out = 2.f * en - 0.5f * (float)np * ush;
    w_out = 12.f * (c2.vir.x + c2.vir.y);
    force[i] = make_float4(-24.f * (c2.fx.x + c2.fx.y), -24.f * (c2.fy.x + c2.fy.y), -24.f * (c2.fz.x + c2.fz.y),
                           e_out);
  }
  if (part) warp_partials3<float>(e_out, w_out, np, part, nwarp);
}

// ----------------------------------------------------------------------------
// Flattened kernel (one type, FP32): the same culled walk, split in two.  The
// warp first walks its rows in lockstep (the rows are the same for all lanes
// up to the cutoff), and each lane only records its non-empty in-grid
// segments [j0, j1) in its own column of a shared-memory table.  The lanes
// then run one packed pair loop each over the concatenation of their
// segments, all for the same number of iterations (the largest lane's), so a
// lane whose window in one row is short goes straight on to its next row
// instead of idling until the longest window of that row ends.  Segments that
// reach a periodic image are evaluated afterwards by the lanes that have them,
// with the exact image shifts of the row walk.  When some lane's column could
// overflow, the table is drained before the walk goes on.
// ----------------------------------------------------------------------------
constexpr int kFlatCap = 24;  // table entries per lane

__global__ void __launch_bounds__(kForceBlock) k_forces_flat(int64_t n, const float4* __restrict__ pos,
                                                             const float* __restrict__ rc,
                                                             const int32_t* __restrict__ start,
                                                             ForceArgs<float> a, float4* __restrict__ force,
                                                             double* __restrict__ part, int64_t nwarp) {
  __shared__ int2 table[kForceBlock / 32][kFlatCap][32];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int2 (*tab)[32] = table[threadIdx.x >> 5];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n;
  const Grid<float>& g = a.g;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const float l = g.edge, il = g.inv_edge, ilx = g.inv_edge_x;
  const float4 pi = valid ? __ldg(pos + i) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float rci = clamp_cutoff<float>(valid ? __ldg(rc + i) : 0.f, a.rc_max);
  const float rc2 = rci * rci, rc2s = rc2 * 1.000004f;
  const int cx = cell_coord<float>(pi.x, g.edge_x, ilx, nx), cy = cell_coord<float>(pi.y, l, il, ny),
            cz = cell_coord<float>(pi.z, l, il, nz);
  const int H = valid ? (int)ceilf(rci * il) : -1, Hx = valid ? (int)ceilf(rci * ilx) : -1;
  int Hw = H;
  for (int o = 16; o > 0; o >>= 1) Hw = max(Hw, __shfl_xor_sync(FULL, Hw, o));
  const int self = (int)i;
  Acc2 c2;
  int cnt = 0, iters = 0;  // table entries, packed iterations they need
  bool img = false;        // some segment reaches a periodic image
  const int side = 2 * Hw + 1, nrows = side * side;
  int dz = -Hw, dy = -Hw;
  for (int r = 0; r <= nrows; ++r) {
    if (r == nrows || __any_sync(FULL, cnt > kFlatCap - 2)) {
      // drain: every lane runs the warp's largest iteration count
      int T = iters;
      for (int o = 16; o > 0; o >>= 1) T = max(T, __shfl_xor_sync(FULL, T, o));
      int k = 0, j = 0, je = 0;
      int2 nxt = cnt > 0 ? tab[0][lane] : make_int2(0, 0);
      for (int it = 0; it < T; ++it) {
        if (j >= je && k < cnt) {
          j = nxt.x;
          je = nxt.y;
          if (++k < cnt) nxt = tab[k][lane];
        }
        const bool v0 = j < je, v1 = j + 1 < je;
        const float4 p0 = __ldg(pos + (v0 ? j : 0)), p1 = __ldg(pos + (v1 ? j + 1 : 0));
        pair_x2<false>(p0, p1, v0, v1, pi.x, pi.y, pi.z, 0.f, 0.f, 0.f, rc2, c2);
        j += 2;
      }
      cnt = 0;
      iters = 0;
      if (r == nrows) break;
    }
    const int uz = cz + dz, uy = cy + dy;
    const float gz = uz > cz ? (float)uz * l - pi.z : (uz < cz ? pi.z - (float)(uz + 1) * l : 0.f);
    const float gy = uy > cy ? (float)uy * l - pi.y : (uy < cy ? pi.y - (float)(uy + 1) * l : 0.f);
    const float gyz2 = gz * gz + gy * gy;
    if (dz >= -H && dz <= H && dy >= -H && dy <= H && gyz2 < rc2s) {
      const float wx = window_half_width(rc2s - gyz2);
      const int ulo = max(ufloor<float>((pi.x - wx) * ilx - 5e-4f), cx - Hx);
      const int uhi = min(ufloor<float>((pi.x + wx) * ilx + 5e-4f), cx + Hx);
      const bool img_row = uy < 0 || uy >= ny || uz < 0 || uz >= nz;
      img |= img_row || ulo < 0 || uhi >= nx;
      const int a0 = max(ulo, 0), a1 = min(uhi, nx - 1);
      if (!img_row && a0 <= a1) {
        const int64_t row = (int64_t)nx * (uy + (int64_t)ny * uz);
        const int j0 = __ldg(start + row + a0), j1 = __ldg(start + row + a1 + 1);
        auto push = [&](int s0, int s1) {
          if (s0 < s1) {
            tab[cnt][lane] = make_int2(s0, s1);
            ++cnt;
            iters += (s1 - s0 + 1) >> 1;
          }
        };
        if (dz == 0 && dy == 0) {  // the particle's own row: cut it out
          push(j0, min(j1, self));
          push(max(j0, self + 1), j1);
        } else {
          push(j0, j1);
        }
      }
    }
    if (++dy > Hw) {
      dy = -Hw;
      ++dz;
    }
  }
  if (img) {
    Acc<float> c;
    const float zero[4] = {0.f, 0.f, 0.f, 0.f};
    walk_rows<float, false, true, Walk::kImagesOnly>(pos, start, g, a, self, pi, rci, 0, zero, c, c2);
  }
  float e_out = 0.f, w_out = 0.f;
  int np = c2.np;
  if (valid) {
    float ush = 0.f;
    if (a.shift && rc2 > 0.f) {
      const float s2 = 1.f / rc2, s6 = s2 * s2 * s2;
      ush = 4.f * s6 * (s6 - 1.f);
    }
    e_out = 2.f * (c2.en.x + c2.en.y) - 0.5f * (float)np * ush;
    w_out = 12.f * (c2.vir.x + c2.vir.y);
    force[i] = make_float4(-24.f * (c2.fx.x + c2.fx.y), -24.f * (c2.fy.x + c2.fy.y), -24.f * (c2.fz.x + c2.fz.y),
                           e_out);
  }
  if (part) warp_partials3<float>(e_out, w_out, np, part, nwarp);
}

// ----------------------------------------------------------------------------
// Two-phase force kernel (one type, FP32, eps = sigma = 1): every lane first
// filters its candidates row by row and appends the accepted ones (r_ij and
// r^2) to its own shared-memory buffer; before a row whose window could
// overflow any lane's buffer, and at the end, the warp drains all buffers
// together and only then does the pair arithmetic.  Rejected candidates (about
// two thirds with cell-granular windows) cost a distance test instead of the
// whole pair evaluation.
// ----------------------------------------------------------------------------
constexpr int kBuf = 32;      // accepted pairs buffered per lane
constexpr int kF2Block = 128;

__device__ __forceinline__ void drain(const float4 (*buf)[kF2Block], int cnt, Acc<float>& c) {
  for (int k = 0; k < cnt; ++k) {
    float4 e = buf[k][threadIdx.x];
    float inv = recip(e.w);
    float s6 = inv * inv * inv;
    float pv = s6 * fmaf(2.0f, s6, -1.0f);
    float q = pv * inv;
    c.fx = fmaf(q, e.x, c.fx);
    c.fy = fmaf(q, e.y, c.fy);
    c.fz = fmaf(q, e.z, c.fz);
    c.en += fmaf(s6, s6, -s6);
    c.vir += pv;
  }
  c.np += cnt;
}

template <bool SJ>
__device__ __forceinline__ int filter_range(const float4* __restrict__ pos, int lo, int hi, float xi, float yi,
                                            float zi, float shx, float shy, float shz, float rc2,
                                            float4 (*buf)[kF2Block], int cnt) {
  for (int j = lo; j < hi; ++j) {
    float4 pj = __ldg(pos + j);
    float dx, dy, dz;
    if (SJ) {
      dx = xi - (pj.x + shx);
      dy = yi - (pj.y + shy);
      dz = zi - (pj.z + shz);
    } else {
      dx = xi - pj.x;
      dy = yi - pj.y;
      dz = zi - pj.z;
    }
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < rc2) {
      buf[cnt][threadIdx.x] = make_float4(dx, dy, dz, r2);
      ++cnt;
    }
  }
  return cnt;
}

__global__ void __launch_bounds__(kF2Block) k_forces2(int64_t n, const float4* __restrict__ pos,
                                                      const float* __restrict__ rc, const int32_t* __restrict__ start,
                                                      ForceArgs<float> a, float4* __restrict__ force,
                                                      double* __restrict__ part, int64_t nwarp) {
  __shared__ float4 buf[kBuf][kF2Block];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  Acc<float> c;
  int cnt = 0;
  float e_out = 0.f, w_out = 0.f;
  const Grid<float>& g = a.g;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const float l = g.edge, il = g.inv_edge, ilx = g.inv_edge_x;
  float4 pi = live ? __ldg(pos + i) : make_float4(0.f, 0.f, 0.f, 0.f);
  float rci = live ? rc[i] : 0.f;
  if (!(rci <= a.rc_max)) rci = a.rc_max;
  if (!(rci > 0.f)) rci = 0.f;
  const float rc2 = rci * rci;
  const float rc2s = rc2 * 1.000004f;
  const int cx = cell_coord<float>(pi.x, g.edge_x, ilx, nx);
  const int cy = cell_coord<float>(pi.y, l, il, ny);
  const int cz = cell_coord<float>(pi.z, l, il, nz);
  const int H = live ? (int)ceilf(rci * il) : -1, Hx = live ? (int)ceilf(rci * ilx) : -1;
  // the warp walks the union of its lanes' (dz, dy) rows in lockstep
  int Hw = H;
  for (int o = 16; o > 0; o >>= 1) Hw = max(Hw, __shfl_xor_sync(0xffffffffu, Hw, o));
  const int self = (int)i;
  for (int dz = -Hw; dz <= Hw; ++dz) {
    int uz = cz + dz;
    float gz = uz > cz ? (float)uz * l - pi.z : (uz < cz ? pi.z - (float)(uz + 1) * l : 0.f);
    float gz2 = gz * gz;
    int wz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
    float zi = uz >= nz ? pi.z - g.L[2] : pi.z;
    float zsh = uz < 0 ? -g.L[2] : 0.f;
    for (int dy = -Hw; dy <= Hw; ++dy) {
      int uy = cy + dy;
      float gy = uy > cy ? (float)uy * l - pi.y : (uy < cy ? pi.y - (float)(uy + 1) * l : 0.f);
      float gyz2 = gz2 + gy * gy;
      bool on = dz >= -H && dz <= H && dy >= -H && dy <= H && gyz2 < rc2s;
      int ulo = 0, uhi = -1;
      int64_t row = 0;
      float yi = pi.y, ysh = 0.f;
      if (on) {
        int wy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
        yi = uy >= ny ? pi.y - g.L[1] : pi.y;
        ysh = uy < 0 ? -g.L[1] : 0.f;
        float wx = window_half_width(rc2s - gyz2);
        ulo = max((int)floorf((pi.x - wx) * ilx - 5e-4f), cx - Hx);
        uhi = min((int)floorf((pi.x + wx) * ilx + 5e-4f), cx + Hx);
        row = (int64_t)nx * (wy + (int64_t)ny * wz);
      }
      // the candidates this row can add: the three pieces of the window (the
      // part before x = 0, the in-grid part, the part past x = L), exactly
      // the ranges filtered below
      int wlen = 0;
      if (on && ulo <= uhi) {
        if (ulo < 0) wlen += __ldg(start + row + min(uhi, -1) + nx + 1) - __ldg(start + row + ulo + nx);
        const int m0 = max(ulo, 0), m1 = min(uhi, nx - 1);
        if (m0 <= m1) wlen += __ldg(start + row + m1 + 1) - __ldg(start + row + m0);
        if (uhi >= nx) wlen += __ldg(start + row + uhi - nx + 1) - __ldg(start + row + max(ulo, nx) - nx);
      }
      if (__any_sync(0xffffffffu, cnt + wlen > kBuf)) {
        drain(buf, cnt, c);
        cnt = 0;
      }
      if (!on || ulo > uhi) continue;
      if (wlen > kBuf) {
        // a window longer than the buffer (very dense or very wide rows): evaluate in place
        for (int seg = 0; seg < 3; ++seg) {
          int s0, s1;
          float xi = pi.x, xsh = 0.f;
          if (seg == 0) { s0 = ulo; s1 = min(uhi, -1); xsh = -g.L[0]; }
          else if (seg == 1) { s0 = max(ulo, 0); s1 = min(uhi, nx - 1); }
          else { s0 = max(ulo, nx); s1 = uhi; xi = pi.x - g.L[0]; }
          if (s0 > s1) continue;
          int w0 = seg == 0 ? s0 + nx : (seg == 2 ? s0 - nx : s0);
          int w1 = seg == 0 ? s1 + nx : (seg == 2 ? s1 - nx : s1);
          int j0 = __ldg(start + row + w0), j1 = __ldg(start + row + w1 + 1);
          pair_range<float, true, false>(pos, j0, min(j1, self), xi, yi, zi, xsh, ysh, zsh, rc2, 0, a, nullptr, c);
          pair_range<float, true, false>(pos, max(j0, self + 1), j1, xi, yi, zi, xsh, ysh, zsh, rc2, 0, a, nullptr, c);
        }
        continue;
      }
      if (ulo < 0) {
        int s1 = min(uhi, -1);
        cnt = filter_range<true>(pos, __ldg(start + row + ulo + nx), __ldg(start + row + s1 + nx + 1), pi.x, yi, zi,
                                 -g.L[0], ysh, zsh, rc2, buf, cnt);
      }
      {
        int s0 = max(ulo, 0), s1 = min(uhi, nx - 1);
        if (s0 <= s1) {
          int j0 = __ldg(start + row + s0), j1 = __ldg(start + row + s1 + 1);
          if (ysh == 0.f && zsh == 0.f) {
            cnt = filter_range<false>(pos, j0, min(j1, self), pi.x, yi, zi, 0.f, 0.f, 0.f, rc2, buf, cnt);
            cnt = filter_range<false>(pos, max(j0, self + 1), j1, pi.x, yi, zi, 0.f, 0.f, 0.f, rc2, buf, cnt);
          } else {
            cnt = filter_range<true>(pos, j0, j1, pi.x, yi, zi, 0.f, ysh, zsh, rc2, buf, cnt);
          }
        }
      }
      if (uhi >= nx) {
        int s0 = max(ulo, nx);
        cnt = filter_range<true>(pos, __ldg(start + row + s0 - nx), __ldg(start + row + uhi - nx + 1),
                                 pi.x - g.L[0], yi, zi, 0.f, ysh, zsh, rc2, buf, cnt);
      }
    }
  }
  drain(buf, cnt, c);
  if (live) {
    float ush = 0.f;
    if (a.shift) {
      float s2 = 1.f / rc2, s6 = s2 * s2 * s2;
      ush = 4.f * s6 * (s6 - 1.f);
    }
    e_out = 2.f * c.en - 0.5f * (float)c.np * ush;
    w_out = 12.f * c.vir;
    force[i] = make_float4(24.f * c.fx, 24.f * c.fy, 24.f * c.fz, e_out);
  }
  if (part) warp_partials3<float>(e_out, w_out, c.np, part, nwarp);
}

// Kernels 2 to 5 serve one-type mixed-precision runs with eps = sigma = 1;
// kernel 3 also serves mixed runs of one or two types with their own eps and
// sigma (its typed packed loop).
int resolve_force_kernel(const dcm_ctx* ctx) {
  int k = force_kernel_choice(ctx->p);
  if (k == DCM_FORCE_THREAD) return k;
  if (ctx->p.precision != DCM_PREC_MIXED) return DCM_FORCE_THREAD;
  const LJTable t = lj_table(ctx->p);
  if (lj_general(t)) return k == DCM_FORCE_PACKED && t.ntypes <= 2 ? k : DCM_FORCE_THREAD;
  return k;
}

template <typename R>
int lj_forces(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc, const int32_t* cell_start,
              typename RT<R>::R4* force, double* totals, cudaStream_t st) {
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
  int64_t nblk = (n + kForceBlock - 1) / kForceBlock;
  int64_t nwarp = nblk * (kForceBlock / 32);
  if (totals && nwarp > ctx->red_cap)
    return set_error(ctx, DCM_ERR_CAPACITY, "force reduction needs %lld partials", (long long)nwarp);
  double* part = totals ? ctx->red : nullptr;
  auto kern = lj_general(t) ? k_forces<R, true> : k_forces<R, false>;
  stage_begin(ctx, DCM_STAGE_FORCES, st);
  bool done = false;
  if constexpr (sizeof(R) == 4) {
    const ForceArgs<float>& af = a;
    const int kind = resolve_force_kernel(ctx);
    if (kind == DCM_FORCE_FLAT) {
      DCM_LAUNCH(ctx, k_forces_flat, (unsigned)nblk, kForceBlock, 0, st, n, pos, rc, cell_start, af, force, part,
                 nwarp);
      done = true;
    } else if (kind == DCM_FORCE_TILE) {
      static_assert(32 * kTileWarps == kForceBlock, "partials layout assumes equal blocks");
      DCM_LAUNCH(ctx, k_forces_tile, (unsigned)nblk, kForceBlock, 0, st, n, pos, rc, cell_start, af, force, part,
                 nwarp);
      done = true;
    } else if (kind == DCM_FORCE_PACKED && lj_general(t)) {
      const int64_t nblk2 = (n + kX2Block - 1) / kX2Block;
      nwarp = nblk2 * (kX2Block / 32);
      DCM_LAUNCH(ctx, k_forces_x2t, (unsigned)nblk2, kX2Block, 0, st, n, pos, rc, cell_start, af, force, part, nwarp);
      done = true;
    } else if (kind == DCM_FORCE_PACKED) {
      const int64_t nblk2 = (n + kX2Block - 1) / kX2Block;  // no more warps than the 128-thread grid
      nwarp = nblk2 * (kX2Block / 32);
      DCM_LAUNCH(ctx, k_forces_x2, (unsigned)nblk2, kX2Block, 0, st, n, pos, rc, cell_start, af, force, part, nwarp);
      done = true;
    } else if (kind == DCM_FORCE_TWO_PHASE) {
      static_assert(kF2Block == kForceBlock, "partials layout assumes equal blocks");
      DCM_LAUNCH(ctx, k_forces2, (unsigned)nblk, kF2Block, 0, st, n, pos, rc, cell_start, af, force, part, nwarp);
      done = true;
    }
  }
  if (!done) DCM_LAUNCH(ctx, kern, (unsigned)nblk, kForceBlock, 0, st, n, pos, rc, cell_start, a, force, part, nwarp);
  stage_end(ctx, DCM_STAGE_FORCES, st);
  int r = check_launch(ctx, "lj_forces");
  if (r) return r;
  if (totals) return reduce_partials(ctx, part, nwarp, 3, totals, false, st);
  return DCM_OK;
}

template int lj_forces<float>(dcm_ctx*, int64_t, const float4*, const float*, const int32_t*, float4*, double*,
                              cudaStream_t);
template int lj_forces<double>(dcm_ctx*, int64_t, const dvec4*, const double*, const int32_t*, dvec4*, double*,
                               cudaStream_t);

}  // namespace dcm
