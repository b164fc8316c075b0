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
// zeroes every term.  The per-particle sums follow dcm_params.accumulation
// (plain FP32, FP32 row-segment sums carried in FP64 or with Kahan
// compensation, or every pair term compensated or in FP64); E and W are
// reduced in FP64.
#include <algorithm>
#include <climits>
#include <cmath>

#include "forces_core.cuh"
#include "tile_order.cuh"

namespace dcm {

// Per-warp partial sums of (E, W, pairs): summed across the warp in FP64,
// then stored as one FP64 partial per warp; no block barrier, so warps that
// finish early do not wait.
__device__ __forceinline__ void warp_partials3(double a, double b, int c, double* part, int64_t nslot,
                                               int64_t w) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    part[w] = a;
    part[nslot + w] = b;
    part[2 * nslot + w] = (double)c;
  }
}

// The scalar loop: one candidate per instruction (FP64 form, and FP32 runs
// of three or four types).
template <typename R, bool TYPED, Accum M>
__global__ void __launch_bounds__(kForceBlock) k_forces(int64_t n, const typename RT<R>::R4* __restrict__ pos,
                                                        const R* __restrict__ rc, const int32_t* __restrict__ start,
                                                        ForceArgs<R> a, typename RT<R>::R4* __restrict__ force,
                                                        double* __restrict__ part, int64_t nwarp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e_out = 0, w_out = 0;
  int np = 0;
  if (i < n)
    force[i] = force_one<R, TYPED, false, M>(pos, start, a.g, a, (int)i, ldg4(pos + i), rc[i], e_out, w_out, np);
  if (part) warp_partials3(e_out, w_out, np, part, nwarp, i >> 5);
}

// The same walk with the packed two-candidates-per-instruction pair loop
// (FP32; one type with eps = sigma = 1, or with TYPED one or two types with
// their own eps and sigma).  Blocks of two warps: a block retires only when
// its slowest warp is done, and the row windows of neighbouring particles
// differ, so small blocks keep the SMs fuller (measured: 64 threads 0.4%
// faster than 128, 32 threads 3% and 1024 threads 14% slower).  The plain
// form fits 64 registers (16 blocks per SM); the compensated forms keep five
// more sums per thread and get 80 (12 blocks).
constexpr int kX2Block = 64;
template <Accum M>
constexpr int x2_min_blocks() { return (M == Accum::kPlain || plane_form(M)) ? 16 : 12; }

template <bool TYPED, Accum M, bool EW>
__global__ void __launch_bounds__(kX2Block, x2_min_blocks<M>()) k_forces_x2(int64_t n, const float4* __restrict__ pos,
                                                                          const float* __restrict__ rc,
                                                                          const int32_t* __restrict__ start,
                                                                          ForceArgs<float> a,
                                                                          float4* __restrict__ force,
                                                                          double* __restrict__ part, int64_t nwarp,
                                                                          const int32_t* __restrict__ order) {
  const int64_t i = (int64_t)(order ? __ldg(order + blockIdx.x) : (int32_t)blockIdx.x) * kX2Block + threadIdx.x;
  double e_out = 0, w_out = 0;
  int np = 0;
  if (i < n)
    force[i] = force_one<float, TYPED, true, M, true, EW>(pos, start, a.g, a, (int)i, __ldg(pos + i), rc[i], e_out, w_out,
                                                         np);
  if (part) warp_partials3(e_out, w_out, np, part, nwarp, i >> 5);
}

// The packed kernel serves mixed-precision runs of one or two types; the
// scalar kernel everything else.
int resolve_force_kernel(const dcm_ctx* ctx) {
  int k = force_kernel_choice(ctx->p);
  if (k == DCM_FORCE_THREAD) return k;
  if (ctx->p.precision != DCM_PREC_MIXED) return DCM_FORCE_THREAD;
  const LJTable t = lj_table(ctx->p);
  return t.ntypes <= 2 ? DCM_FORCE_PACKED : DCM_FORCE_THREAD;
}

// The accumulation form a force launch of this context runs (DCM_ACC_*,
// AUTO resolved to the plane-Kahan form, measured the cheapest compensated
// form at the accuracy of the FP64 ones; the FP64 precision form is plain
// FP64; the scalar FP32 kernel runs the row form of a pair form).
int resolve_accumulation(const dcm_ctx* ctx) {
  if (ctx->p.precision != DCM_PREC_MIXED) return DCM_ACC_FP32;
  int m = ctx->p.accumulation == DCM_ACC_AUTO ? DCM_ACC_PLANE_KAHAN : ctx->p.accumulation;
  if (resolve_force_kernel(ctx) != DCM_FORCE_PACKED) {
    if (m == DCM_ACC_PAIR_KAHAN) m = DCM_ACC_ROW_KAHAN;
    if (m == DCM_ACC_PAIR_FP64) m = DCM_ACC_ROW_FP64;
  }
  return m;
}

namespace {

// Cost key of the packed kernel's tiles (tile_order.cuh): the largest cutoff
// among a tile's particles.
__global__ void __launch_bounds__(kX2Block) k_force_tile_key(int64_t n, const float* __restrict__ rc, float rc_max,
                                                             int32_t* __restrict__ key, int32_t* __restrict__ cnt,
                                                             int64_t nchunk) {
  const int64_t i = (int64_t)blockIdx.x * kX2Block + threadIdx.x;
  tile_key_of_block(i < n ? clamp_cutoff<float>(__ldg(rc + i), rc_max) : 0.f, rc_max, key, cnt, nchunk);
}

template <Accum M>
int launch_x2(dcm_ctx* ctx, bool typed, bool ew, int64_t n, const float4* pos, const float* rc,
               const int32_t* cell_start, const ForceArgs<float>& a, float4* force, double* part, int64_t nwarp,
               cudaStream_t st) {
  const unsigned nblk = (unsigned)((n + kX2Block - 1) / kX2Block);
  // launch order of the tiles, the widest walks first, where the launch is
  // short enough for that to pay
  const int32_t* order = nullptr;
  if (tile_order_pays((const void*)k_forces_x2<false, M, false>, kX2Block, nblk)) {
    const TileOrder to = tile_order_layout(ctx->tile_scratch, nblk);
    int r = tile_order_begin(ctx, to, st);
    if (r) return r;
    DCM_LAUNCH(ctx, k_force_tile_key, nblk, kX2Block, 0, st, n, rc, a.rc_max, to.key, to.cnt, to.nchunk);
    if ((r = tile_order_finish(ctx, to, st))) return r;
    order = to.order;
  }
  if (typed && ew)
    DCM_LAUNCH(ctx, (k_forces_x2<true, M, true>), nblk, kX2Block, 0, st, n, pos, rc, cell_start, a, force, part, nwarp,
               order);
  else if (typed)
    DCM_LAUNCH(ctx, (k_forces_x2<true, M, false>), nblk, kX2Block, 0, st, n, pos, rc, cell_start, a, force, part,
               nwarp, order);
  else if (ew)
    DCM_LAUNCH(ctx, (k_forces_x2<false, M, true>), nblk, kX2Block, 0, st, n, pos, rc, cell_start, a, force, part,
               nwarp, order);
  else
    DCM_LAUNCH(ctx, (k_forces_x2<false, M, false>), nblk, kX2Block, 0, st, n, pos, rc, cell_start, a, force, part,
               nwarp, order);
  return DCM_OK;
}

template <typename R, Accum M>
void launch_scalar(dcm_ctx* ctx, bool typed, int64_t n, const typename RT<R>::R4* pos, const R* rc,
                   const int32_t* cell_start, const ForceArgs<R>& a, typename RT<R>::R4* force, double* part,
                   int64_t nwarp, cudaStream_t st) {
  const unsigned nblk = (unsigned)((n + kForceBlock - 1) / kForceBlock);
  if (typed)
    DCM_LAUNCH(ctx, (k_forces<R, true, M>), nblk, kForceBlock, 0, st, n, pos, rc, cell_start, a, force, part, nwarp);
  else
    DCM_LAUNCH(ctx, (k_forces<R, false, M>), nblk, kForceBlock, 0, st, n, pos, rc, cell_start, a, force, part,
               nwarp);
}

}  // namespace

template <typename R>
int lj_forces(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc, const int32_t* cell_start,
              typename RT<R>::R4* force, double* totals, cudaStream_t st, bool energies) {
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
  const bool typed = lj_general(t);
  const int kind = resolve_force_kernel(ctx);
  const int block = kind == DCM_FORCE_PACKED ? kX2Block : kForceBlock;
  const int64_t nwarp = (n + block - 1) / block * (block / 32);
  if (totals && nwarp > ctx->red_cap)
    return set_error(ctx, DCM_ERR_CAPACITY, "force reduction needs %lld partials", (long long)nwarp);
  double* part = totals ? ctx->red : nullptr;
  stage_begin(ctx, DCM_STAGE_FORCES, st);
  if constexpr (sizeof(R) == 4) {
    const int m = resolve_accumulation(ctx);
    if (kind == DCM_FORCE_PACKED) {
      const int r = with_accum<true>(m, [&](auto tag) {
        return launch_x2<decltype(tag)::value>(ctx, typed, energies || totals, n, pos, rc, cell_start, a, force, part,
                                               nwarp, st);
      });
      if (r) return r;
    } else
      with_accum<false>(m, [&](auto tag) {
        launch_scalar<float, decltype(tag)::value>(ctx, typed, n, pos, rc, cell_start, a, force, part, nwarp, st);
        return 0;
      });
  } else {
    launch_scalar<R, Accum::kPlain>(ctx, typed, n, pos, rc, cell_start, a, force, part, nwarp, st);
  }
  stage_end(ctx, DCM_STAGE_FORCES, st);
  int r = check_launch(ctx, "lj_forces");
  if (r) return r;
  if (totals) return reduce_partials(ctx, part, nwarp, 3, totals, false, st);
  return DCM_OK;
}

template int lj_forces<float>(dcm_ctx*, int64_t, const float4*, const float*, const int32_t*, float4*, double*,
                              cudaStream_t, bool);
template int lj_forces<double>(dcm_ctx*, int64_t, const dvec4*, const double*, const int32_t*, dvec4*, double*,
                               cudaStream_t, bool);

}  // namespace dcm
