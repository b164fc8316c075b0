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
