// Velocity-Verlet timestep around the DCM pipeline (Section 2; Fig. 3).
//
//   kick-drift-count:  v += dt/2 F;  x += dt v (wrapped);  cell and provisional
//                      rank of every particle (atomic count)        [fused]
//   scan, scatter, per-cell stable sort, gather into the other buffer
//   every K steps:     box counts -> interface -> distances -> cutoffs
//   forces;  kick:     v += dt/2 F with the kinetic energy reduced in FP64
#include <algorithm>

#include "dcm_internal.cuh"

namespace dcm {

template <typename R>
__device__ __forceinline__ R wrap_coord(R x, R L) {
  if (x >= L) x -= L;
  if (x < (R)0) {
    x += L;
    if (x >= L) x = (R)0;  // a tiny negative value rounded up to L
  }
  return x;
}

// kicks = 1: the first half kick of a step; kicks = 2: also the second half
// kick of the previous step (the same two roundings as two launches), used
// inside a multi-step call where that step's kinetic energy is not reported.
template <typename R>
__global__ void k_kick_drift_count(int64_t n, typename RT<R>::R4* __restrict__ pos, typename RT<R>::R4* __restrict__ vel,
                                   const typename RT<R>::R4* __restrict__ force, R half_dt, R dt, Grid<R> g,
                                   int32_t* __restrict__ cell, int32_t* __restrict__ slot, int32_t* __restrict__ count,
                                   int kicks) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto p = pos[i];
  auto v = vel[i];
  auto f = force[i];
  for (int k = 0; k < kicks; ++k) {
    v.x += half_dt * f.x;
    v.y += half_dt * f.y;
    v.z += half_dt * f.z;
  }
  p.x = wrap_coord<R>(p.x + dt * v.x, g.L[0]);
  p.y = wrap_coord<R>(p.y + dt * v.y, g.L[1]);
  p.z = wrap_coord<R>(p.z + dt * v.z, g.L[2]);
  pos[i] = p;
  vel[i] = v;
  int cx = cell_coord<R>(p.x, g.edge_x, g.inv_edge_x, g.n[0]);
  int cy = cell_coord<R>(p.y, g.edge, g.inv_edge, g.n[1]);
  int cz = cell_coord<R>(p.z, g.edge, g.inv_edge, g.n[2]);
  int c = cx + g.n[0] * (cy + g.n[1] * cz);
  cell[i] = c;
  slot[i] = atomicAdd(count + c, 1);
}

// Second half kick and kinetic energy: per-thread and per-warp sums in the
// working precision, one FP64 partial per warp.
template <typename R>
__global__ void k_kick_ke(int64_t n, typename RT<R>::R4* __restrict__ vel, const typename RT<R>::R4* __restrict__ force,
                          R half_dt, double* __restrict__ part) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  R ke = 0;
  if (i < n) {
    auto v = vel[i];
    if (force) {
      auto f = force[i];
      v.x += half_dt * f.x;
      v.y += half_dt * f.y;
      v.z += half_dt * f.z;
      vel[i] = v;
    }
    ke = (R)0.5 * (v.x * v.x + v.y * v.y + v.z * v.z);
  }
  for (int o = 16; o > 0; o >>= 1) ke += __shfl_xor_sync(0xffffffffu, ke, o);
  if ((threadIdx.x & 31) == 0) part[i >> 5] = (double)ke;
}

// One pass over perm for the whole particle payload.
template <typename R>
__global__ void k_gather_state(int64_t n, const int32_t* __restrict__ perm, const typename RT<R>::R4* __restrict__ p0,
                               typename RT<R>::R4* __restrict__ p1, const typename RT<R>::R4* __restrict__ v0,
                               typename RT<R>::R4* __restrict__ v1, const R* __restrict__ r0, R* __restrict__ r1,
                               const int32_t* __restrict__ id0, int32_t* __restrict__ id1) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int src = perm[k];
  p1[k] = p0[src];
  v1[k] = v0[src];
  r1[k] = r0[src];
  if (id0) id1[k] = id0[src];
}

__global__ void k_thermo(const double* totals, double* thermo) {
  thermo[0] = totals[0];  // E
  thermo[1] = totals[1];  // W
  thermo[2] = totals[3];  // KE
  thermo[3] = totals[2];  // accepted pairs
}

template <typename R>
static int recompute_cutoffs(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, R* rc, cudaStream_t st) {
  const int32_t* box_count;
  int r;
  if (ctx->p.h == ctx->p.l && ctx->p.lx == ctx->p.l) {
    box_count = ctx->cell_count;  // the binning's counts are the gray-scale volume's input
  } else {
    r = histogram<R>(ctx, n, pos, box_grid<R>(ctx), ctx->box_count, st);
    if (r) return r;
    box_count = ctx->box_count;
  }
  stage_begin(ctx, DCM_STAGE_DETECT, st);
  r = detect_interface(ctx, box_count, ctx->s, ctx->iface, nullptr, nullptr, st);
  stage_end(ctx, DCM_STAGE_DETECT, st);
  if (r) return r;
  stage_begin(ctx, DCM_STAGE_DISTANCE, st);
  r = distance_sweeps<R>(ctx, ctx->s, ctx->iface, (R*)ctx->D[0], nullptr, false, st);
  stage_end(ctx, DCM_STAGE_DISTANCE, st);
  if (r) return r;
  stage_begin(ctx, DCM_STAGE_CUTOFFS, st);
  r = assign_cutoffs<R>(ctx, n, pos, (const R*)ctx->D[0], rc, st);
  stage_end(ctx, DCM_STAGE_CUTOFFS, st);
  return r;
}

template <typename R>
static int finish_thermo(dcm_ctx* ctx, int64_t n, typename RT<R>::R4* vel, const typename RT<R>::R4* force, R half_dt,
                         double* thermo, cudaStream_t st) {
  int64_t nblk = (n + 255) / 256, nwarp = nblk * 8;
  if (nwarp > ctx->red_cap) return set_error(ctx, DCM_ERR_CAPACITY, "kinetic reduction too large");
  if (n > 0) {
    DCM_LAUNCH(ctx, k_kick_ke<R>, (unsigned)nblk, 256, 0, st, n, vel, force, half_dt, ctx->red);
    int r = reduce_partials(ctx, ctx->red, nwarp, 1, ctx->totals + 3, false, st);
    if (r) return r;
  } else {
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->totals + 3, 0, sizeof(double), st));
  }
  if (thermo) DCM_LAUNCH(ctx, k_thermo, 1, 1, 0, st, ctx->totals, thermo);
  return check_launch(ctx, "thermo");
}

template <typename R>
static int gather_state(dcm_ctx* ctx, dcm_state* st, int64_t n, cudaStream_t s) {
  using R4 = typename RT<R>::R4;
  int c = st->cur, o = 1 - st->cur;
  bool ids = st->id[c] && st->id[o];
  if (n > 0)
    DCM_LAUNCH(ctx, k_gather_state<R>, (unsigned)((n + 255) / 256), 256, 0, s, n, ctx->perm, (const R4*)st->pos[c],
               (R4*)st->pos[o], (const R4*)st->vel[c], (R4*)st->vel[o], (const R*)st->rc[c], (R*)st->rc[o],
               ids ? st->id[c] : nullptr, ids ? st->id[o] : nullptr);
  return check_launch(ctx, "gather_state");
}

template <typename R>
int step_init(dcm_ctx* ctx, dcm_state* st, int64_t n, cudaStream_t s) {
  using R4 = typename RT<R>::R4;
  int o = 1 - st->cur;
  Grid<R> g = cell_grid<R>(ctx);
  int r = bin_particles<R>(ctx, n, (const R4*)st->pos[st->cur], g, ctx->cell, ctx->cell_start, ctx->perm, nullptr, s);
  if (r) return r;
  if ((r = gather_state<R>(ctx, st, n, s))) return r;
  if ((r = recompute_cutoffs<R>(ctx, n, (const R4*)st->pos[o], (R*)st->rc[o], s))) return r;
  if (ctx->p.skin > 0.0) {
    if ((r = list_build<R>(ctx, n, (const R4*)st->pos[o], (const R*)st->rc[o], s))) return r;
    r = list_forces<R>(ctx, n, (const R4*)st->pos[o], (const R*)st->rc[o], (R4*)st->force, ctx->totals, s);
  } else {
    r = lj_forces<R>(ctx, n, (const R4*)st->pos[o], (const R*)st->rc[o], ctx->cell_start, (R4*)st->force,
                     ctx->totals, s);
  }
  if (r) return r;
  if ((r = finish_thermo<R>(ctx, n, (R4*)st->vel[o], nullptr, (R)0, st->thermo, s))) return r;
  st->cur = o;
  st->t = 0;
  return DCM_OK;
}

// Steps with Verlet lists: rebin and rebuild only when needed.
template <typename R>
static int step_run_lists(dcm_ctx* ctx, dcm_state* st, int64_t n, double dt, int nsteps, cudaStream_t s) {
  using R4 = typename RT<R>::R4;
  Grid<R> g = cell_grid<R>(ctx);
  R hdt = (R)(0.5 * dt), rdt = (R)dt;
  int K = ctx->p.recompute_every;
  for (int k = 0; k < nsteps; ++k) {
    int r;
    bool recompute = (st->t + 1) % K == 0;
    bool rebuild = recompute || !ctx->list_valid;
    // as in step_run: only the last step of the call reports thermo, the
    // others' second half kick rides on the next step's kick-drift launch
    const bool last = k == nsteps - 1;
    const int kicks = k == 0 ? 1 : 2;
    stage_begin(ctx, DCM_STAGE_KICK_DRIFT, s);
    if (rebuild) {
      DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cell_count, 0, sizeof(int32_t) * ctx->ncell, s));
      if (n > 0)
        DCM_LAUNCH(ctx, k_kick_drift_count<R>, (unsigned)((n + 255) / 256), 256, 0, s, n, (R4*)st->pos[st->cur],
                   (R4*)st->vel[st->cur], (const R4*)st->force, hdt, rdt, g, ctx->cell, ctx->slot, ctx->cell_count,
                   kicks);
    } else {
      if ((r = list_kick_drift<R>(ctx, st, n, hdt, rdt, kicks, &rebuild, s))) return r;
      if (rebuild && (r = list_wrap_count<R>(ctx, st, n, s))) return r;
    }
    stage_end(ctx, DCM_STAGE_KICK_DRIFT, s);
    st->t += 1;
    if (rebuild) {
      int o = 1 - st->cur;
      stage_begin(ctx, DCM_STAGE_BIN, s);
      if ((r = exclusive_scan(ctx, ctx->cell_count, ctx->cell_start, ctx->ncell, s))) return r;
      if ((r = scatter_sort(ctx, n, ctx->cell, ctx->slot, ctx->cell_start, ctx->ncell, ctx->perm, s))) return r;
      if ((r = gather_state<R>(ctx, st, n, s))) return r;
      stage_end(ctx, DCM_STAGE_BIN, s);
      if (recompute)
        if ((r = recompute_cutoffs<R>(ctx, n, (const R4*)st->pos[o], (R*)st->rc[o], s))) return r;
      if ((r = list_build<R>(ctx, n, (const R4*)st->pos[o], (const R*)st->rc[o], s))) return r;
      st->cur = o;
    }
    int c = st->cur;
    if ((r = list_forces<R>(ctx, n, (const R4*)st->pos[c], (const R*)st->rc[c], (R4*)st->force,
                            last ? ctx->totals : nullptr, s, last)))
      return r;
    if (last) {
      stage_begin(ctx, DCM_STAGE_KICK, s);
      if ((r = finish_thermo<R>(ctx, n, (R4*)st->vel[c], (const R4*)st->force, hdt, st->thermo, s))) return r;
      stage_end(ctx, DCM_STAGE_KICK, s);
    }
  }
  return DCM_OK;
}

template <typename R>
int step_run(dcm_ctx* ctx, dcm_state* st, int64_t n, double dt, int nsteps, cudaStream_t s) {
  using R4 = typename RT<R>::R4;
  if (ctx->p.skin > 0.0) return step_run_lists<R>(ctx, st, n, dt, nsteps, s);
  Grid<R> g = cell_grid<R>(ctx);
  R hdt = (R)(0.5 * dt), rdt = (R)dt;
  int K = ctx->p.recompute_every;
  for (int k = 0; k < nsteps; ++k) {
    int c = st->cur, o = 1 - c;
    // only the last step of the call reports thermo: the second half kick of
    // the others is applied by the next step's kick-drift launch
    const bool last = k == nsteps - 1;
    stage_begin(ctx, DCM_STAGE_KICK_DRIFT, s);
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cell_count, 0, sizeof(int32_t) * ctx->ncell, s));
    if (n > 0)
      DCM_LAUNCH(ctx, k_kick_drift_count<R>, (unsigned)((n + 255) / 256), 256, 0, s, n, (R4*)st->pos[c],
                 (R4*)st->vel[c], (const R4*)st->force, hdt, rdt, g, ctx->cell, ctx->slot, ctx->cell_count,
                 k == 0 ? 1 : 2);
    stage_end(ctx, DCM_STAGE_KICK_DRIFT, s);
    stage_begin(ctx, DCM_STAGE_BIN, s);
    int r = exclusive_scan(ctx, ctx->cell_count, ctx->cell_start, ctx->ncell, s);
    if (r) return r;
    if ((r = scatter_sort(ctx, n, ctx->cell, ctx->slot, ctx->cell_start, ctx->ncell, ctx->perm, s))) return r;
    if ((r = gather_state<R>(ctx, st, n, s))) return r;
    stage_end(ctx, DCM_STAGE_BIN, s);
    st->t += 1;
    if (st->t % K == 0)
      if ((r = recompute_cutoffs<R>(ctx, n, (const R4*)st->pos[o], (R*)st->rc[o], s))) return r;
    // energy and virial only where they are reported (the call's last step)
    if ((r = lj_forces<R>(ctx, n, (const R4*)st->pos[o], (const R*)st->rc[o], ctx->cell_start, (R4*)st->force,
                          last ? ctx->totals : nullptr, s, last)))
      return r;
    if (last) {
      stage_begin(ctx, DCM_STAGE_KICK, s);
      if ((r = finish_thermo<R>(ctx, n, (R4*)st->vel[o], (const R4*)st->force, hdt, st->thermo, s))) return r;
      stage_end(ctx, DCM_STAGE_KICK, s);
    }
    st->cur = o;
  }
  return DCM_OK;
}

template int step_init<float>(dcm_ctx*, dcm_state*, int64_t, cudaStream_t);
template int step_init<double>(dcm_ctx*, dcm_state*, int64_t, cudaStream_t);
template int step_run<float>(dcm_ctx*, dcm_state*, int64_t, double, int, cudaStream_t);
template int step_run<double>(dcm_ctx*, dcm_state*, int64_t, double, int, cudaStream_t);

}  // namespace dcm
