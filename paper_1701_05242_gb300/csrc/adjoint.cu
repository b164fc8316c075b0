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
                                                            const int32_t* __restrict__ bmax) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int np = a.ntypes * a.ntypes;
  AdjAcc<R> c;
  for (int p = 0; p < 16; ++p) c.de[p] = c.ds[p] = (R)0;
  if (i < n) {
    const Grid<R>& g = a.g;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const R l = g.edge, il = g.inv_edge, ilx = g.inv_edge_x;
    auto pi = ldg4(pos + i);
    auto ak = ldg4(A + i);
    R rck = rc[i];
    if (!(rck <= a.rc_max)) rck = a.rc_max;
    if (!(rck > (R)0)) rck = (R)0;
    const R rck2 = rck * rck;
    R reach = a.rc_max;  // reverse pairs: the largest cutoff around k
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
          adj_range<R, TYPED>(pos, rc, A, __ldg(start + row + ulo + nx), __ldg(start + row + a1 + nx + 1), -1, pi.x,
                              yi, zi, -g.L[0], ysh, zsh, rck2, tk, ak, half_dlde, a, ku, kd, c);
        }
        {
          int a0 = max(ulo, 0), a1 = min(uhi, nx - 1);
          if (a0 <= a1)
            adj_range<R, TYPED>(pos, rc, A, __ldg(start + row + a0), __ldg(start + row + a1 + 1),
                                (ysh == (R)0 && zsh == (R)0) ? (int)i : -1, pi.x, yi, zi, (R)0, ysh, zsh, rck2, tk, ak,
                                half_dlde, a, ku, kd, c);
        }
        if (uhi >= nx) {
          int a0 = max(ulo, nx);
          adj_range<R, TYPED>(pos, rc, A, __ldg(start + row + a0 - nx), __ldg(start + row + uhi - nx + 1), -1,
                              pi.x - g.L[0], yi, zi, (R)0, ysh, zsh, rck2, tk, ak, half_dlde, a, ku, kd, c);
        }
      }
    }
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
  auto kern = lj_general(t) ? k_adjoint<R, true> : k_adjoint<R, false>;
  DCM_LAUNCH(ctx, kern, (unsigned)nblk, kBlock, 0, st, n, pos, rc, cell_start, a, A, (R)(0.5 * dlde), G, part,
             nwarp, bg, (const int32_t*)ctx->blk_max);
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
