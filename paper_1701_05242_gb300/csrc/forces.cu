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

// unwrapped cell index (no clamp) of a coordinate, used only for culling
template <typename R>
__device__ __forceinline__ int ufloor(R v) {
  return (int)floor(v);
}

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
  R fx = 0, fy = 0, fz = 0, en = 0, vir = 0;
  int npair = 0;
  if (i < n) {
    const Grid<R>& g = a.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const R l = g.edge, il = g.inv_edge;
    auto pi = ldg4(pos + i);
    // cutoffs outside [0, rc_max] (or NaN) are clamped: the stencil then never
    // reaches past one periodic image, which keeps every cell index in range
    R rci = rc[i];
    if (!(rci <= a.rc_max)) rci = a.rc_max;
    if (!(rci > (R)0)) rci = (R)0;
    const R rc2 = rci * rci;
    const R rc2s = rc2 * (R)1.000004;  // culling slack; the pair test below is exact
    const int ti = TYPED ? type_of(pi.w, a.ntypes) : 0;
    R ushift[4] = {0, 0, 0, 0};
    if (a.shift) {
      for (int t = 0; t < (TYPED ? a.ntypes : 1); ++t) {
        int tp = ti * a.ntypes + t;
        R s2 = (TYPED ? a.sig2[tp] : (R)1) / rc2;
        R s6 = s2 * s2 * s2;
        ushift[t] = (TYPED ? a.eps4[tp] : (R)4) * s6 * (s6 - (R)1);
      }
    }
    const int cx = cell_coord<R>(pi.x, l, il, nx);
    const int cy = cell_coord<R>(pi.y, l, il, ny);
    const int cz = cell_coord<R>(pi.z, l, il, nz);
    const int H = (int)ceil(rci * il);
    for (int uz = cz - H; uz <= cz + H; ++uz) {
      R gz = uz > cz ? (R)uz * l - pi.z : (uz < cz ? pi.z - (R)(uz + 1) * l : (R)0);
      R gz2 = gz * gz;
      if (gz2 >= rc2s) continue;
      int wz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
      R zi = uz >= nz ? pi.z - g.L[2] : pi.z;       // image +L: shift i
      R zsh = uz < 0 ? -g.L[2] : (R)0;               // image -L: shift j
      for (int uy = cy - H; uy <= cy + H; ++uy) {
        R gy = uy > cy ? (R)uy * l - pi.y : (uy < cy ? pi.y - (R)(uy + 1) * l : (R)0);
        R gyz2 = gz2 + gy * gy;
        if (gyz2 >= rc2s) continue;
        int wy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
        R yi = uy >= ny ? pi.y - g.L[1] : pi.y;
        R ysh = uy < 0 ? -g.L[1] : (R)0;
        R wx = sqrt(rc2s - gyz2);
        int ulo = ufloor<R>((pi.x - wx) * il - (R)5e-4);
        int uhi = ufloor<R>((pi.x + wx) * il + (R)5e-4);
        ulo = max(ulo, cx - H);
        uhi = min(uhi, cx + H);
        const int64_t row = (int64_t)nx * (wy + (int64_t)ny * wz);
        // up to three segments: u < 0 (image -L), 0 <= u < nx, u >= nx (image +L)
#pragma unroll 1
        for (int seg = 0; seg < 3; ++seg) {
          int a0, a1;
          R xi, xsh;
          if (seg == 0) {
            a0 = ulo;
            a1 = min(uhi, -1);
            xi = pi.x;
            xsh = -g.L[0];
          } else if (seg == 1) {
            a0 = max(ulo, 0);
            a1 = min(uhi, nx - 1);
            xi = pi.x;
            xsh = (R)0;
          } else {
            a0 = max(ulo, nx);
            a1 = uhi;
            xi = pi.x - g.L[0];
            xsh = (R)0;
          }
          if (a0 > a1) continue;
          int w0 = seg == 0 ? a0 + nx : (seg == 2 ? a0 - nx : a0);
          int w1 = seg == 0 ? a1 + nx : (seg == 2 ? a1 - nx : a1);
          int j0 = __ldg(start + row + w0), j1 = __ldg(start + row + w1 + 1);
          for (int j = j0; j < j1; ++j) {
            auto pj = ldg4(pos + j);
            R dx = xi - (pj.x + xsh);
            R dy = yi - (pj.y + ysh);
            R dz = zi - (pj.z + zsh);
            R r2 = fma(dx, dx, fma(dy, dy, dz * dz));
            bool acc = (r2 < rc2) && (j != (int)i);
            R inv = recip(r2);
            inv = acc ? inv : (R)0;
            R s2, e24, e4, us;
            if (TYPED) {
              int tj = type_of(pj.w, a.ntypes);
              int tp = ti * a.ntypes + tj;
              s2 = a.sig2[tp] * inv;
              e24 = a.eps24[tp];
              e4 = a.eps4[tp];
              us = tj == 0 ? ushift[0] : (tj == 1 ? ushift[1] : (tj == 2 ? ushift[2] : ushift[3]));
            } else {
              s2 = inv;
              e24 = (R)24;
              e4 = (R)4;
              us = ushift[0];
            }
            R s6 = s2 * s2 * s2;
            R pv = e24 * s6 * fma((R)2, s6, (R)-1);  // r . F_ij
            R fs = pv * inv;
            fx = fma(fs, dx, fx);
            fy = fma(fs, dy, fy);
            fz = fma(fs, dz, fz);
            R u = e4 * s6 * (s6 - (R)1);
            en += acc ? u - us : (R)0;
            vir += pv;
            npair += acc ? 1 : 0;
          }
        }
      }
    }
    typename RT<R>::R4 out;
    out.x = fx;
    out.y = fy;
    out.z = fz;
    out.w = (R)0.5 * en;
    force[i] = out;
  }
  if (part) warp_partials3<R>((R)0.5 * en, (R)0.5 * vir, npair, part, nwarp);
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
  auto kern = t.ntypes > 1 ? k_forces<R, true> : k_forces<R, false>;
  stage_begin(ctx, DCM_STAGE_FORCES, st);
  DCM_LAUNCH(ctx, kern, (unsigned)nblk, kForceBlock, 0, st, n, pos, rc, cell_start, a, force, part, nwarp);
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
