// Batched form: R independent systems (replicas) of different sizes stepped
// together.  Two launch plans share the per-element device code of
// batch_core.cuh:
//   - the persistent plan (default): two cooperative launches per timestep
//     that run every stage, with bounded grid-wide barriers between them and
//     the force stage pulling (replica, tile) work items from a device queue
//     (batch_persist.cu);
//   - the per-stage plan: each stage one launch over the concatenation of all
//     replicas (this file).
// The whole K-step recomputation period can be captured once in a CUDA graph
// and replayed (dcm_batch_capture / dcm_batch_replay): every size is fixed,
// the distance sweeps run inside one cooperative launch until a sweep
// changes nothing (at most iter_max), and no call inside a step waits on the
// host.
#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstring>
#include <new>
#include <vector>

#include "batch_core.cuh"
#include "grid_sync.cuh"
#include "tile_order.cuh"

namespace dcm {

static int berr(dcm_batch* b, int code, const char* fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->base.err, sizeof(b->base.err), fmt, ap);
    va_end(ap);
  }
  return code;
}

// ---- per-stage kernels (one thread per element) ----------------------------------
template <typename R>
__global__ void k_b_kick_drift_count(int64_t n, typename RT<R>::R4* __restrict__ pos, typename RT<R>::R4* __restrict__ vel,
                                     const typename RT<R>::R4* __restrict__ force, R half_dt, R dt, R l, R il,
                                     R lx, R ilx, const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep,
                                     int32_t* __restrict__ cell, int32_t* __restrict__ slot, int32_t* __restrict__ count,
                                     int drift) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b_kick_drift_count<R>(i, pos, vel, force, half_dt, dt, l, il, lx, ilx, geom, rep, cell, slot, count, drift);
}

template <typename R>
__global__ void k_b_gather(int64_t n, const int32_t* __restrict__ perm, const typename RT<R>::R4* __restrict__ p0,
                           typename RT<R>::R4* __restrict__ p1, const typename RT<R>::R4* __restrict__ v0,
                           typename RT<R>::R4* __restrict__ v1, const R* __restrict__ r0, R* __restrict__ r1,
                           const int32_t* __restrict__ id0, int32_t* __restrict__ id1) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) b_gather<R>(k, perm, p0, p1, v0, v1, r0, r1, id0, id1);
}

template <typename R>
__global__ void k_b_box_count(int64_t n, const typename RT<R>::R4* __restrict__ pos, R h, R ih,
                              const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep,
                              int32_t* __restrict__ count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b_box_count<R>(i, pos, h, ih, geom, rep, count);
}

template <int AXIS>
__global__ void k_b_box_sum(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t nbox,
                            const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep, int w) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbox) b_box_sum<AXIS>(b, in, out, geom, rep, w);
}

__global__ void k_b_thr_init(int32_t* thr, int R, int fixed) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < R) b_thr_init(r, thr, fixed);
}

__global__ void k_b_minmax(const int32_t* __restrict__ g, int64_t nbox, const uint16_t* __restrict__ rep, int32_t* thr) {
  b_minmax((int64_t)blockIdx.x * blockDim.x + threadIdx.x, g, nbox, rep, thr);
}

__global__ void k_b_value_hist(const int32_t* __restrict__ g, int64_t nbox, const uint16_t* __restrict__ rep,
                               const int32_t* thr, int32_t* hist, int32_t* status) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbox) b_value_hist(b, g, rep, thr, hist, status);
}

// one block per replica
__global__ void k_b_two_means(const int32_t* __restrict__ hist, int32_t* thr, int max_iter) {
  b_two_means(blockIdx.x, hist, thr, max_iter);
}

__global__ void k_b_segment(const int32_t* __restrict__ g, int64_t nbox, const RepGeom* __restrict__ geom,
                            const uint16_t* __restrict__ rep, const int32_t* thr, uint8_t* __restrict__ s,
                            uint8_t* __restrict__ iface) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbox) b_segment(b, g, geom, rep, thr, s, iface);
}

template <typename R>
__global__ void k_b_dist_init(const uint8_t* __restrict__ s, const uint8_t* __restrict__ iface, int64_t nbox,
                              R* __restrict__ D0, R* __restrict__ D1) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbox) b_dist_init<R>(b, s, iface, D0, D1);
}

// All Jacobi sweeps of every replica in one cooperative launch (every block
// resident): a bounded grid barrier after each sweep, until a sweep changes
// nothing or `budget` sweeps have run (the same iterates as one launch per
// sweep).  A barrier wait past budget_ns records DCM_ERR_TIMEOUT.
template <typename R>
__global__ void __launch_bounds__(256) k_b_dist_coop(R* D0, R* D1, int64_t nbox, const RepGeom* __restrict__ geom,
                                                     const uint16_t* __restrict__ rep, R h, R r_grid, int32_t* flags,
                                                     int budget, uint32_t* sync, int64_t budget_ns, int32_t* status) {
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  for (int it = 0; it < budget; ++it) {
    if (it > 0 && ((volatile int32_t*)flags)[it - 1] == 0) break;  // the previous sweep changed nothing
    const R* Din = (it & 1) ? D1 : D0;
    R* Dout = (it & 1) ? D0 : D1;
    bool changed = false;
    for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x; k0 < nbox; k0 += gs) {
      const int64_t k = k0 + threadIdx.x;
      if (k < nbox) changed |= b_dist_update<R, true>(k, Din, Dout, geom, rep, h, r_grid);
    }
    if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) flags[it] = 1;
    if (!grid_sync(sync, gridDim.x, budget_ns, status)) return;
  }
}

__global__ void k_b_dist_finish(const int32_t* flags, int sweeps, int32_t* status) {
  int first = -1;
  for (int k = 0; k < sweeps; ++k)
    if (flags[k] == 0) {
      first = k;
      break;
    }
  if (first < 0) raise_status(status, DCM_ERR_NOT_CONVERGED);
}

template <typename R>
__global__ void k_b_cutoffs(int64_t n, const typename RT<R>::R4* __restrict__ pos, const R* __restrict__ D,
                            const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep, R h, R r_grid,
                            R rc_min, R rc_max, R ramp, R* __restrict__ rc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b_cutoffs<R>(i, pos, D, geom, rep, h, r_grid, rc_min, rc_max, ramp, rc);
}

template <typename R, bool TYPED, bool X2, Accum M, bool EW = true>
__global__ void k_b_forces(int64_t n, const typename RT<R>::R4* __restrict__ pos, const R* __restrict__ rc,
                           const int32_t* __restrict__ start, ForceArgs<R> a, const RepGeom* __restrict__ geom,
                           const uint16_t* __restrict__ rep, typename RT<R>::R4* __restrict__ force,
                           R* __restrict__ w_i, int32_t* __restrict__ np_i, const int32_t* __restrict__ order) {
  const int64_t i = (int64_t)(order ? __ldg(order + blockIdx.x) : (int32_t)blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) b_force<R, TYPED, X2, M, true, EW>(i, pos, rc, start, a, geom, rep, force, w_i, np_i);
}

// Cost key of the force tiles (tile_order.cuh): the largest cutoff among a
// tile's particles.
template <typename R>
__global__ void k_b_tile_key(int64_t n, const R* __restrict__ rc, R rc_max, int32_t* __restrict__ key,
                             int32_t* __restrict__ cnt, int64_t nchunk) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  tile_key_of_block(i < n ? (float)clamp_cutoff<R>(rc[i], rc_max) : 0.f, (float)rc_max, key, cnt, nchunk);
}

template <typename R>
__global__ void k_b_kick(int64_t n, typename RT<R>::R4* __restrict__ vel, const typename RT<R>::R4* __restrict__ force,
                         R half_dt, R* __restrict__ ke_i) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b_kick<R>(i, vel, force, half_dt, ke_i);
}

// Per-replica thermo in two fixed-order levels: one block per chunk of at
// most kThermoChunk particles of one replica (FP64 sums), then one warp per
// replica over its chunks.  thermo[4 r + {0,1,2,3}] = {E, W, KE, pairs}.
template <typename R>
__global__ void k_b_thermo_chunks(const int64_t* __restrict__ chunk, int32_t nchunk,
                                  const typename RT<R>::R4* __restrict__ force, const R* __restrict__ w_i,
                                  const R* __restrict__ ke_i, const int32_t* __restrict__ np_i,
                                  double* __restrict__ tpart) {
  b_thermo_chunk<R>(blockIdx.x, chunk, nchunk, force, w_i, ke_i, np_i, tpart);
}

__global__ void k_b_thermo_sum(const int32_t* __restrict__ chunk0, int R, int32_t nchunk,
                               const double* __restrict__ tpart, double* __restrict__ thermo) {
  const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (r < R) b_thermo_sum(r, chunk0, nchunk, tpart, thermo);
}

// ---- orchestration ------------------------------------------------------------------
template <typename R>
static int b_recompute(dcm_batch* b, const typename RT<R>::R4* pos, R* rc, cudaStream_t st) {
  dcm_ctx* ctx = &b->base;
  const dcm_params& p = b->p;
  int64_t n = b->ntot, nb = b->nbox_tot;
  unsigned gp = (unsigned)((n + 255) / 256), gb = (unsigned)((nb + 255) / 256);
  const int32_t* counts = ctx->cell_count;
  if (p.h != p.l || p.lx != p.l) {
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->box_count, 0, sizeof(int32_t) * nb, st));
    if (n > 0)
      DCM_LAUNCH(ctx, k_b_box_count<R>, gp, 256, 0, st, n, pos, (R)p.h, (R)(1.0 / p.h), b->geom, b->rep_of_particle,
                 ctx->box_count);
    counts = ctx->box_count;
  }
  stage_begin(ctx, DCM_STAGE_DETECT, st);
  int w = p.smooth_w;
  DCM_LAUNCH(ctx, k_b_box_sum<0>, gb, 256, 0, st, counts, ctx->g, nb, b->geom, b->rep_of_box, w);
  DCM_LAUNCH(ctx, k_b_box_sum<1>, gb, 256, 0, st, ctx->g, ctx->g_tmp, nb, b->geom, b->rep_of_box, w);
  DCM_LAUNCH(ctx, k_b_box_sum<2>, gb, 256, 0, st, ctx->g_tmp, ctx->g, nb, b->geom, b->rep_of_box, w);
  DCM_LAUNCH(ctx, k_b_thr_init, (unsigned)((b->R + 63) / 64), 64, 0, st, b->thr, b->R, p.threshold);
  if (p.threshold < 0) {
    DCM_LAUNCH(ctx, k_b_minmax, gb, 256, 0, st, ctx->g, nb, b->rep_of_box, b->thr);
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(b->hist, 0, sizeof(int32_t) * (size_t)b->R * kBatchHistBins, st));
    DCM_LAUNCH(ctx, k_b_value_hist, gb, 256, 0, st, ctx->g, nb, b->rep_of_box, b->thr, b->hist, ctx->status);
    DCM_LAUNCH(ctx, k_b_two_means, (unsigned)b->R, 1024, 0, st, b->hist, b->thr, 64);
  }
  DCM_LAUNCH(ctx, k_b_segment, gb, 256, 0, st, ctx->g, nb, b->geom, b->rep_of_box, b->thr, ctx->s, ctx->iface);
  stage_end(ctx, DCM_STAGE_DETECT, st);
  stage_begin(ctx, DCM_STAGE_DISTANCE, st);
  R* D0 = (R*)ctx->D[0];
  R* D1 = (R*)ctx->D[1];
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->flags, 0, sizeof(int32_t) * (size_t)(p.iter_max + 2), st));
  DCM_LAUNCH(ctx, k_b_dist_init<R>, gb, 256, 0, st, ctx->s, ctx->iface, nb, D0, D1);
  // every sweep in one cooperative launch, until one changes nothing or the
  // even budget iter_max (rounded up) runs out
  const int budget = p.iter_max + (p.iter_max & 1);
  {
    auto kern = k_b_dist_coop<R>;
    int per_sm = 0, sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1)
      return set_error(ctx, DCM_ERR_CUDA, "batch distance sweeps: occupancy query failed");
    const unsigned grid =
        (unsigned)std::min<int64_t>((int64_t)std::min(per_sm, 4) * sms, std::max<int64_t>((nb + 255) / 256, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->coop_sync, 0, 4 * sizeof(uint32_t), st));
    ++ctx->launches;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, D0, D1, nb, (const RepGeom*)b->geom, (const uint16_t*)b->rep_of_box,
                                       (R)p.h, (R)p.r_grid, ctx->flags, budget, ctx->coop_sync, (int64_t)2000000000,
                                       ctx->status);
    if (e != cudaSuccess) return set_error(ctx, DCM_ERR_CUDA, "batch distance sweeps: %s", cudaGetErrorString(e));
  }
  DCM_LAUNCH(ctx, k_b_dist_finish, 1, 1, 0, st, ctx->flags, budget, ctx->status);
  stage_end(ctx, DCM_STAGE_DISTANCE, st);
  stage_begin(ctx, DCM_STAGE_CUTOFFS, st);
  if (n > 0)
    DCM_LAUNCH(ctx, k_b_cutoffs<R>, gp, 256, 0, st, n, pos, D0, b->geom, b->rep_of_particle, (R)p.h, (R)p.r_grid,
               (R)p.rc_min, (R)p.rc_max, (R)p.ramp, rc);
  stage_end(ctx, DCM_STAGE_CUTOFFS, st);
  return check_launch(ctx, "batch recompute");
}

template <typename R>
ForceArgs<R> batch_force_args(const dcm_batch* b) {
  ForceArgs<R> a;
  a.g.edge = (R)b->p.l;
  a.g.inv_edge = (R)(1.0 / b->p.l);
  a.g.edge_x = (R)b->p.lx;
  a.g.inv_edge_x = (R)(1.0 / b->p.lx);
  LJTable t = lj_table(b->p);
  a.ntypes = t.ntypes;
  for (int k = 0; k < 16; ++k) {
    a.eps24[k] = (R)t.deps24[k];
    a.eps4[k] = (R)t.deps4[k];
    a.sig2[k] = (R)t.dsig2[k];
  }
  a.shift = b->p.shift_energy;
  a.rc_max = (R)b->p.rc_max;
  return a;
}
template ForceArgs<float> batch_force_args<float>(const dcm_batch*);
template ForceArgs<double> batch_force_args<double>(const dcm_batch*);

// The batched force kernel for the LJ table and the accumulation form
// (DCM_ACC_*, resolved as for a single system; the batched form runs the
// plain and plane forms, and the plane form of the other compensated ones).
int batch_accumulation(const dcm_batch* b) {
  const int m = resolve_accumulation(&b->base);
  if (m == DCM_ACC_FP32) return m;
  return (m == DCM_ACC_ROW_FP64 || m == DCM_ACC_PAIR_FP64 || m == DCM_ACC_PLANE_FP64) ? DCM_ACC_PLANE_FP64
                                                                                      : DCM_ACC_PLANE_KAHAN;
}

template <typename R>
static auto b_force_kernel(bool typed, int ntypes, int acc, bool energies) {
  using K = void (*)(int64_t, const typename RT<R>::R4*, const R*, const int32_t*, ForceArgs<R>, const RepGeom*,
                     const uint16_t*, typename RT<R>::R4*, R*, int32_t*, const int32_t*);
  if constexpr (sizeof(R) == 8) {
    return typed ? (K)k_b_forces<R, true, false, Accum::kPlain> : (K)k_b_forces<R, false, false, Accum::kPlain>;
  } else {
    const bool x2 = !(typed && ntypes > 2);
    auto pick = [&](auto tag) -> K {
      constexpr Accum M = decltype(tag)::value;
      if (!x2) return (K)k_b_forces<R, true, false, M>;  // the scalar loop always sums energy and virial
      if (energies) return typed ? (K)k_b_forces<R, true, true, M> : (K)k_b_forces<R, false, true, M>;
      return typed ? (K)k_b_forces<R, true, true, M, false> : (K)k_b_forces<R, false, true, M, false>;
    };
    if (acc == DCM_ACC_FP32) return pick(AccumTag<Accum::kPlain>{});
    if (acc == DCM_ACC_PLANE_FP64) return pick(AccumTag<Accum::kPlaneF64>{});
    return pick(AccumTag<Accum::kPlaneKahan>{});
  }
}

template <typename R>
// Forces, second half kick and (with energies) the per-replica thermo; without
// energies the timestep's forces alone (a timestep whose thermo nothing reads).
static int b_forces_thermo(dcm_batch* b, const typename RT<R>::R4* pos, const R* rc, typename RT<R>::R4* force,
                           typename RT<R>::R4* vel, R half_dt, bool kick, double* thermo, cudaStream_t st,
                           bool energies = true) {
  dcm_ctx* ctx = &b->base;
  int64_t n = b->ntot;
  if (n > 0) {
    const ForceArgs<R> a = batch_force_args<R>(b);
    const LJTable t = lj_table(b->p);
    int bs = b->force_block;
    // the packed loop in FP32 for one type, and for one or two types with
    // their own eps and sigma; the scalar loop otherwise
    auto kern = b_force_kernel<R>(lj_general(t), t.ntypes, batch_accumulation(b), energies);
    stage_begin(ctx, DCM_STAGE_FORCES, st);
    const TileOrder to = tile_order_layout(ctx->tile_scratch, (n + bs - 1) / bs);
    const int32_t* order = nullptr;  // the widest tiles first, where that pays
    if (tile_order_pays((const void*)kern, bs, to.ntile)) {
      int r = tile_order_begin(ctx, to, st);
      if (r) return r;
      DCM_LAUNCH(ctx, k_b_tile_key<R>, (unsigned)to.ntile, bs, 0, st, n, rc, a.rc_max, to.key, to.cnt, to.nchunk);
      if ((r = tile_order_finish(ctx, to, st))) return r;
      order = to.order;
    }
    DCM_LAUNCH(ctx, kern, (unsigned)to.ntile, bs, 0, st, n, pos, rc, ctx->cell_start, a, b->geom,
               b->rep_of_particle, force, (R*)b->w_i, b->np_i, order);
    stage_end(ctx, DCM_STAGE_FORCES, st);
    stage_begin(ctx, DCM_STAGE_KICK, st);
    DCM_LAUNCH(ctx, k_b_kick<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, vel, kick ? force : nullptr, half_dt,
               energies ? (R*)b->ke_i : nullptr);
    if (energies) {
      if (b->nchunk > 0)
        DCM_LAUNCH(ctx, k_b_thermo_chunks<R>, (unsigned)b->nchunk, 256, 0, st, b->chunk, b->nchunk, force,
                   (const R*)b->w_i, (const R*)b->ke_i, b->np_i, b->tpart);
      DCM_LAUNCH(ctx, k_b_thermo_sum, (unsigned)((b->R + 7) / 8), 256, 0, st, b->chunk0, b->R, b->nchunk, b->tpart,
                 thermo);
    }
    stage_end(ctx, DCM_STAGE_KICK, st);
  }
  return check_launch(ctx, "batch forces");
}

template <typename R>
static int b_bin_gather(dcm_batch* b, dcm_state* s, bool drift, R hdt, R dt, cudaStream_t st) {
  using R4 = typename RT<R>::R4;
  dcm_ctx* ctx = &b->base;
  int64_t n = b->ntot;
  int c = s->cur, o = 1 - c;
  stage_begin(ctx, DCM_STAGE_KICK_DRIFT, st);
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cell_count, 0, sizeof(int32_t) * b->ncell_tot, st));
  if (n > 0)
    DCM_LAUNCH(ctx, k_b_kick_drift_count<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, (R4*)s->pos[c],
               (R4*)s->vel[c], (const R4*)s->force, hdt, dt, (R)b->p.l, (R)(1.0 / b->p.l), (R)b->p.lx,
               (R)(1.0 / b->p.lx), b->geom,
               b->rep_of_particle, ctx->cell, ctx->slot, ctx->cell_count, drift ? 1 : 0);
  stage_end(ctx, DCM_STAGE_KICK_DRIFT, st);
  stage_begin(ctx, DCM_STAGE_BIN, st);
  int r = exclusive_scan(ctx, ctx->cell_count, ctx->cell_start, b->ncell_tot, st);
  if (r) return r;
  if ((r = scatter_sort(ctx, n, ctx->cell, ctx->slot, ctx->cell_start, b->ncell_tot, ctx->perm, st))) return r;
  bool ids = s->id[c] && s->id[o];
  if (n > 0)
    DCM_LAUNCH(ctx, k_b_gather<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, ctx->perm, (const R4*)s->pos[c],
               (R4*)s->pos[o], (const R4*)s->vel[c], (R4*)s->vel[o], (const R*)s->rc[c], (R*)s->rc[o],
               ids ? s->id[c] : nullptr, ids ? s->id[o] : nullptr);
  stage_end(ctx, DCM_STAGE_BIN, st);
  return check_launch(ctx, "batch bin");
}

template <typename R>
static int b_init(dcm_batch* b, dcm_state* s, cudaStream_t st) {
  using R4 = typename RT<R>::R4;
  if (b->persistent) {
    int r = b_persistent_step<R>(b, s, (R)0, (R)0, false, true, false, true, st);
    if (r) return r;
    s->cur = 1 - s->cur;
    s->t = 0;
    return DCM_OK;
  }
  int r = b_bin_gather<R>(b, s, false, (R)0, (R)0, st);
  if (r) return r;
  int o = 1 - s->cur;
  if ((r = b_recompute<R>(b, (const R4*)s->pos[o], (R*)s->rc[o], st))) return r;
  if ((r = b_forces_thermo<R>(b, (const R4*)s->pos[o], (const R*)s->rc[o], (R4*)s->force, (R4*)s->vel[o], (R)0,
                              false, s->thermo, st)))
    return r;
  s->cur = o;
  s->t = 0;
  return DCM_OK;
}

template <typename R>
static int b_steps(dcm_batch* b, dcm_state* s, double dt, int nsteps, cudaStream_t st) {
  using R4 = typename RT<R>::R4;
  R hdt = (R)(0.5 * dt), rdt = (R)dt;
  int K = b->p.recompute_every;
  for (int k = 0; k < nsteps; ++k) {
    // energy, virial and thermo only on the call's last timestep (the only
    // one whose thermo is read)
    const bool last = k == nsteps - 1;
    if (b->persistent) {
      s->t += 1;
      int r = b_persistent_step<R>(b, s, hdt, rdt, true, s->t % K == 0, true, last, st);
      if (r) return r;
      s->cur = 1 - s->cur;
      continue;
    }
    int r = b_bin_gather<R>(b, s, true, hdt, rdt, st);
    if (r) return r;
    int o = 1 - s->cur;
    s->t += 1;
    if (s->t % K == 0)
      if ((r = b_recompute<R>(b, (const R4*)s->pos[o], (R*)s->rc[o], st))) return r;
    if ((r = b_forces_thermo<R>(b, (const R4*)s->pos[o], (const R*)s->rc[o], (R4*)s->force, (R4*)s->vel[o], hdt,
                                true, s->thermo, st, last)))
      return r;
    s->cur = o;
  }
  return DCM_OK;
}

}  // namespace dcm

using namespace dcm;

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" void dcm_batch_destroy(dcm_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  dcm_ctx* c = &b->base;
  void* dev[] = {c->status, c->coop_sync, c->slot,  c->cell,  c->perm,   c->cell_start, c->cell_count, c->scan_state,
                 c->box_count, c->g,   c->g_tmp, c->s,      c->iface,      c->D[0],       c->D[1],
                 c->flags,  c->red,   c->red_tmp, c->totals, b->geom,       b->rep_of_particle, b->rep_of_box,
                 b->thr,    b->hist,  b->w_i,   b->ke_i,   b->np_i, b->chunk, b->chunk0, b->tpart,
                 b->tiles,  b->sync,  b->scan_blk, b->pacc, c->tile_scratch};
  for (void* q : dev)
    if (q) cudaFree(q);
  if (c->host_status) cudaFreeHost(c->host_status);
  if (c->ev) {
    for (int64_t k = 0; k < (int64_t)DCM_NSTAGES * c->ev_cap * 2; ++k)
      if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    free(c->ev);
  }
  delete b;
}

extern "C" int dcm_batch_create(const dcm_params* p, int32_t R, const double* boxes, const int64_t* counts,
                                dcm_batch** out) {
  if (!p || !boxes || !counts || !out || R < 1 || R > 65535) return DCM_ERR_INVALID_ARG;
  *out = nullptr;
  if (p->skin != 0.0) return DCM_ERR_INVALID_ARG;  // the batched form steps over cell lists only
  if (p->min_component != 0) return DCM_ERR_INVALID_ARG;  // no bubble filter in the batched form
  if (p->segmentation != 0) return DCM_ERR_INVALID_ARG;   // nor the regularised segmentation
  std::vector<RepGeom> geom((size_t)R);
  int64_t ntot = 0, nctot = 0, nbtot = 0;
  for (int r = 0; r < R; ++r) {
    dcm_params q = *p;
    for (int d = 0; d < 3; ++d) q.box[d] = boxes[3 * r + d];
    q.n_max = counts[r];
    int v = dcm_validate_params(&q, nullptr, 0);
    if (v) return v;
    if (counts[r] < 0) return DCM_ERR_INVALID_ARG;
    int64_t nc[3], nb[3];
    dcm_grid_dims(&q, nc, nb);
    RepGeom& G = geom[(size_t)r];
    G.p0 = ntot;
    G.p1 = ntot + counts[r];
    G.c0 = nctot;
    G.b0 = nbtot;
    for (int d = 0; d < 3; ++d) {
      G.nc[d] = (int)nc[d];
      G.nb[d] = (int)nb[d];
      G.L[d] = (double)nc[d] * (d == 0 && p->lx > 0.0 ? p->lx : p->l);
    }
    ntot += counts[r];
    nctot += nc[0] * nc[1] * nc[2];
    nbtot += nb[0] * nb[1] * nb[2];
  }
  if (ntot >= 0x7fffffffLL || nctot >= 0x7fffffffLL || nbtot >= 0x7fffffffLL) return DCM_ERR_CAPACITY;
  dcm_batch* b = new (std::nothrow) dcm_batch();
  if (!b) return DCM_ERR_NOMEM;
  memset(&b->base, 0, sizeof(b->base));
  b->p = *p;
  if (!(b->p.lx > 0.0)) b->p.lx = b->p.l;
  if (!(b->p.ramp > 0.0)) b->p.ramp = b->p.rc_max - b->p.rc_min;
  if (!(b->p.r_grid > 0.0)) b->p.r_grid = b->p.ramp + 2.0 * b->p.h;
  b->R = R;
  b->precision = p->precision;
  b->ntot = ntot;
  b->ncell_tot = nctot;
  b->nbox_tot = nbtot;
  b->geom_h = geom;
  b->geom = nullptr;
  b->rep_of_particle = nullptr;
  b->rep_of_box = nullptr;
  b->thr = nullptr;
  b->hist = nullptr;
  b->w_i = b->ke_i = nullptr;
  b->np_i = nullptr;
  b->nchunk = 0;
  b->chunk = nullptr;
  b->chunk0 = nullptr;
  b->tpart = nullptr;
  b->force_block = 128;
  b->persistent = 1;
  b->tiles = nullptr;
  b->ntiles = 0;
  b->tile = 0;
  b->sync = nullptr;
  b->scan_blk = nullptr;
  b->pacc = nullptr;
  b->pgrid = 0;
  b->wait_budget = (int64_t)2000000000;  // 2 s
  b->graph = nullptr;
  b->graph_steps = 0;
  b->graph_launches = 0;
  memset(b->graph_key, 0, sizeof(b->graph_key));
  dcm_ctx* c = &b->base;
  c->p = b->p;
  c->precision = p->precision;
  c->ncell = nctot;
  c->nbox = nbtot;
  c->n_max = ntot;
  cudaGetDevice(&c->device);
  int64_t rs = p->precision == DCM_PREC_FP64 ? 8 : 4;
  int64_t nm = ntot > 0 ? ntot : 1;
  int64_t big = std::max(nctot, nbtot);
  c->scan_cap = (big + kScanTile - 1) / kScanTile + 1;
  c->red_cap = ((nm + 255) / 256 + 1) * 8;
  bool ok = true;
  auto alloc = [&](void** ptr, int64_t bytes) {
    if (ok && cudaMalloc(ptr, (size_t)(bytes > 0 ? bytes : 16)) != cudaSuccess) ok = false;
  };
  alloc((void**)&c->status, 16);
  alloc((void**)&c->coop_sync, 16);
  alloc((void**)&c->slot, 4 * nm);
  alloc((void**)&c->cell, 4 * nm);
  alloc((void**)&c->perm, 4 * nm);
  alloc((void**)&c->cell_start, 4 * (nctot + 1));
  alloc((void**)&c->cell_count, 4 * nctot);
  alloc((void**)&c->scan_state, 8 * (c->scan_cap + 1));
  alloc((void**)&c->box_count, 4 * nbtot);
  alloc((void**)&c->g, 4 * nbtot);
  alloc((void**)&c->g_tmp, 4 * nbtot);
  alloc((void**)&c->s, nbtot);
  alloc((void**)&c->iface, nbtot);
  alloc(&c->D[0], rs * nbtot);
  alloc(&c->D[1], rs * nbtot);
  alloc((void**)&c->flags, 4 * (int64_t)(p->iter_max + 2));
  alloc((void**)&c->red, 8 * 3 * c->red_cap);
  alloc((void**)&c->red_tmp, 8 * 8 * 256);
  alloc((void**)&c->totals, 8 * 8);
  alloc((void**)&c->tile_scratch, 4 * tile_scratch_ints(nm));
  alloc((void**)&b->geom, (int64_t)sizeof(RepGeom) * R);
  alloc((void**)&b->rep_of_particle, 2 * nm);
  alloc((void**)&b->rep_of_box, 2 * nbtot);
  alloc((void**)&b->thr, 16 * (int64_t)R);
  alloc((void**)&b->hist, 4 * (int64_t)R * kBatchHistBins);
  alloc(&b->w_i, rs * nm);
  alloc(&b->ke_i, rs * nm);
  alloc((void**)&b->np_i, 4 * nm);
  std::vector<int64_t> ch;
  std::vector<int32_t> ch0((size_t)R + 1, 0);
  for (int r = 0; r < R; ++r) {
    ch0[(size_t)r] = (int32_t)(ch.size() / 2);
    for (int64_t a = geom[(size_t)r].p0; a < geom[(size_t)r].p1; a += kThermoChunk) {
      ch.push_back(a);
      ch.push_back(std::min(a + kThermoChunk, geom[(size_t)r].p1));
    }
  }
  b->nchunk = (int32_t)(ch.size() / 2);
  ch0[(size_t)R] = b->nchunk;
  alloc((void**)&b->chunk, 8 * (int64_t)ch.size());
  alloc((void**)&b->chunk0, 4 * ((int64_t)R + 1));
  alloc((void**)&b->tpart, 8 * 4 * (int64_t)std::max<int32_t>(b->nchunk, 1));
  if (ok && cudaMallocHost((void**)&c->host_status, 16) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    dcm_batch_destroy(b);
    return DCM_ERR_NOMEM;
  }
  std::vector<uint16_t> rp((size_t)nm, 0), rb((size_t)(nbtot > 0 ? nbtot : 1), 0);
  for (int r = 0; r < R; ++r) {
    for (int64_t i = geom[r].p0; i < geom[r].p1; ++i) rp[(size_t)i] = (uint16_t)r;
    int64_t nbr = (int64_t)geom[r].nb[0] * geom[r].nb[1] * geom[r].nb[2];
    for (int64_t k = 0; k < nbr; ++k) rb[(size_t)(geom[r].b0 + k)] = (uint16_t)r;
  }
  if (cudaMemcpy(b->geom, geom.data(), sizeof(RepGeom) * R, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->rep_of_particle, rp.data(), 2 * rp.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->rep_of_box, rb.data(), 2 * (size_t)nbtot, cudaMemcpyHostToDevice) != cudaSuccess ||
      (!ch.empty() && cudaMemcpy(b->chunk, ch.data(), 8 * ch.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(b->chunk0, ch0.data(), 4 * ch0.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->status, 0, 16) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    dcm_batch_destroy(b);
    return DCM_ERR_CUDA;
  }
  int ps = b_persistent_setup(b);
  if (ps) {
    cudaGetLastError();
    dcm_batch_destroy(b);
    return ps;
  }
  *out = b;
  return DCM_OK;
}

extern "C" const char* dcm_batch_last_error(const dcm_batch* b) { return b ? b->base.err : "null batch"; }

extern "C" int dcm_batch_offsets(const dcm_batch* b, int64_t* offsets) {
  if (!b || !offsets) return DCM_ERR_INVALID_ARG;
  for (int r = 0; r < b->R; ++r) offsets[r] = b->geom_h[(size_t)r].p0;
  offsets[b->R] = b->ntot;
  return DCM_OK;
}

extern "C" int dcm_batch_set_force_block(dcm_batch* b, int32_t threads) {
  if (!b || (threads != 64 && threads != 128 && threads != 256)) return DCM_ERR_INVALID_ARG;
  b->force_block = threads;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return DCM_OK;
}

static int batch_check_state(dcm_batch* b, const dcm_state* s) {
  if (!s || (s->cur != 0 && s->cur != 1)) return berr(b, DCM_ERR_INVALID_ARG, "bad state");
  if (b->ntot > 0)
    for (int k = 0; k < 2; ++k)
      if (!s->pos[k] || !s->vel[k] || !s->rc[k]) return berr(b, DCM_ERR_INVALID_ARG, "state buffers must be set");
  if (b->ntot > 0 && (!s->force || !s->thermo)) return berr(b, DCM_ERR_INVALID_ARG, "state.force/thermo must be set");
  if ((s->id[0] == nullptr) != (s->id[1] == nullptr)) return berr(b, DCM_ERR_INVALID_ARG, "id needs both buffers");
  return DCM_OK;
}

extern "C" int dcm_batch_step_init(dcm_batch* b, dcm_state* s, dcm_stream_t stream) {
  if (!b) return DCM_ERR_INVALID_ARG;
  int r = batch_check_state(b, s);
  if (r) return r;
  if (b->precision == DCM_PREC_MIXED) return b_init<float>(b, s, (cudaStream_t)stream);
  return b_init<double>(b, s, (cudaStream_t)stream);
}

extern "C" int dcm_batch_step(dcm_batch* b, dcm_state* s, double dt, int32_t nsteps, dcm_stream_t stream) {
  if (!b) return DCM_ERR_INVALID_ARG;
  int r = batch_check_state(b, s);
  if (r) return r;
  if (nsteps < 0 || !(dt > 0.0)) return berr(b, DCM_ERR_INVALID_ARG, "need nsteps >= 0 and dt > 0");
  if (b->precision == DCM_PREC_MIXED) return b_steps<float>(b, s, dt, nsteps, (cudaStream_t)stream);
  return b_steps<double>(b, s, dt, nsteps, (cudaStream_t)stream);
}

extern "C" int dcm_batch_capture(dcm_batch* b, dcm_state* s, double dt, dcm_stream_t stream) {
  if (!b) return DCM_ERR_INVALID_ARG;
  int r = batch_check_state(b, s);
  if (r) return r;
  if (!stream) return berr(b, DCM_ERR_INVALID_ARG, "graph capture needs a non-default stream");
  int K = b->p.recompute_every;
  if (s->t % K != 0) return berr(b, DCM_ERR_INVALID_ARG, "capture must start at a recomputation step (t %% K == 0)");
  if (!(dt > 0.0)) return berr(b, DCM_ERR_INVALID_ARG, "dt must be positive");
  int steps = (K % 2 == 0) ? K : 2 * K;  // even: the double buffers return to the same side
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaStream_t st = (cudaStream_t)stream;
  dcm_state tmp = *s;
  int64_t launches0 = b->base.launches;
  int timing = b->base.timing;
  b->base.timing = 0;  // no event records inside the graph
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return berr(b, DCM_ERR_CUDA, "cudaStreamBeginCapture failed");
  r = (b->precision == DCM_PREC_MIXED) ? b_steps<float>(b, &tmp, dt, steps, st) : b_steps<double>(b, &tmp, dt, steps, st);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  b->base.timing = timing;
  if (r) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (e != cudaSuccess || !graph) return berr(b, DCM_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return berr(b, DCM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  b->graph_steps = steps;
  b->graph_launches = b->base.launches - launches0;
  b->base.launches = launches0;
  void* key[8] = {s->pos[0], s->pos[1], s->vel[0], s->vel[1], s->rc[0], s->rc[1], s->force, s->thermo};
  memcpy(b->graph_key, key, sizeof(key));
  return DCM_OK;
}

extern "C" int dcm_batch_replay(dcm_batch* b, dcm_state* s, int32_t ngraphs, dcm_stream_t stream) {
  if (!b || !s || ngraphs < 0) return DCM_ERR_INVALID_ARG;
  if (!b->graph) return berr(b, DCM_ERR_INVALID_ARG, "no captured graph");
  void* key[8] = {s->pos[0], s->pos[1], s->vel[0], s->vel[1], s->rc[0], s->rc[1], s->force, s->thermo};
  if (memcmp(key, b->graph_key, sizeof(key)) != 0)
    return berr(b, DCM_ERR_INVALID_ARG, "state buffers differ from the captured ones");
  for (int k = 0; k < ngraphs; ++k) {
    cudaError_t e = cudaGraphLaunch(b->graph, (cudaStream_t)stream);
    if (e != cudaSuccess) return berr(b, DCM_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    b->base.launches += b->graph_launches;
    s->t += b->graph_steps;
  }
  return DCM_OK;
}

extern "C" int dcm_batch_graph_steps(const dcm_batch* b) { return b ? b->graph_steps : 0; }

extern "C" int dcm_batch_set_persistent(dcm_batch* b, int32_t on) {
  if (!b || (on != 0 && on != 1)) return DCM_ERR_INVALID_ARG;
  b->persistent = on;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return DCM_OK;
}

extern "C" int dcm_batch_accumulation(const dcm_batch* b, int32_t* form) {
  if (!b || !form) return DCM_ERR_INVALID_ARG;
  *form = b->precision == DCM_PREC_MIXED ? batch_accumulation(b) : DCM_ACC_FP32;
  return DCM_OK;
}

extern "C" int dcm_batch_set_tile(dcm_batch* b, int32_t particles) {
  if (!b) return DCM_ERR_INVALID_ARG;
  int r = b_persistent_set_tile(b, particles);
  if (r) return r;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return DCM_OK;
}

extern "C" int dcm_batch_set_wait_budget(dcm_batch* b, int64_t ns) {
  if (!b || ns < 1000) return DCM_ERR_INVALID_ARG;
  b->wait_budget = ns;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return DCM_OK;
}

extern "C" int dcm_batch_barrier_selftest(dcm_batch* b, int32_t phantom, int64_t budget_ns, dcm_stream_t stream) {
  if (!b || phantom < 0 || budget_ns < 1000 || budget_ns > (int64_t)10000000000) return DCM_ERR_INVALID_ARG;
  return b_persistent_wait_selftest(b, phantom, budget_ns, (cudaStream_t)stream);
}

extern "C" int dcm_batch_status(dcm_batch* b, dcm_stream_t stream) {
  if (!b) return DCM_ERR_INVALID_ARG;
  return dcm_status(&b->base, stream);
}

extern "C" int dcm_batch_set_timing(dcm_batch* b, int32_t capacity) {
  return b ? dcm_set_timing(&b->base, capacity) : DCM_ERR_INVALID_ARG;
}

extern "C" int dcm_batch_stage_times(dcm_batch* b, double* ms, int64_t* count) {
  if (!b) return DCM_ERR_INVALID_ARG;
  double ev_ms[DCM_NSTAGES];
  int64_t ev_n[DCM_NSTAGES];
  int r = dcm_stage_times(&b->base, ev_ms, ev_n);
  // the persistent plan's stage clock (nanoseconds and runs), read and cleared
  unsigned long long acc[2 * DCM_NSTAGES + 1] = {0};
  if (b->pacc) {
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(acc, b->pacc, sizeof(acc), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(b->pacc, 0, sizeof(acc)) != cudaSuccess)
      return berr(b, DCM_ERR_CUDA, "persistent stage clock");
  }
  for (int s = 0; s < DCM_NSTAGES; ++s) {
    if (ms) ms[s] = ev_ms[s] + 1e-6 * (double)acc[s];
    if (count) count[s] = ev_n[s] + (int64_t)acc[DCM_NSTAGES + s];
  }
  return r;
}

extern "C" int dcm_batch_launch_count(dcm_batch* b, int64_t* count, int32_t reset) {
  return b ? dcm_launch_count(&b->base, count, reset) : DCM_ERR_INVALID_ARG;
}
