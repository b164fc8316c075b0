// Batched form, persistent plan: two cooperative launches per timestep run
// every stage of the step for all replicas (Fig. 3's boxes 1-5 inside
// velocity Verlet), with grid-wide barriers between the stages: part 0 the
// half kick, drift, binning and (every K steps) interface, distances and
// cutoffs; part 1 the forces, the second half kick and the per-replica
// thermo.  The split lets part 1 read the positions, cutoffs and cell starts
// that part 0 wrote through the read-only data path (legal only for data no
// thread of the same launch writes); reading them with coherent loads inside
// one launch made the force stage twice as slow.
//
// The grid holds exactly as many blocks as can be resident at once (a
// cooperative launch, which the driver refuses rather than oversubscribe), so
// a barrier never waits for a block that cannot run.  Every barrier wait is
// bounded all the same: a block that polls longer than the batch's wait
// budget records DCM_ERR_TIMEOUT in the device status, raises an abort flag
// and returns, and every other block leaves at its next barrier.
//
// The force stage, which dominates, takes its work from a device queue of
// (replica, tile) items, each 32 consecutive sorted particles of one replica:
// a warp pulls the next item with one atomic and evaluates its particles, so
// replicas of any size and particles of any cutoff spread over the SMs in
// small pieces (the GPU form of the paper's dynamic schedule of 20
// particles per task, Section 2.4).  The other stages run grid-stride loops
// over particles, cells or boxes; the exclusive scan of the cell counts is a
// two-pass block scan (per-block totals, then each block's offset and scan).
#include <algorithm>
#include <climits>
#include <cstring>

#include "batch_core.cuh"
#include "grid_sync.cuh"

namespace dcm {

constexpr int kPBlock = 128;  // threads per block of the persistent kernels
// Blocks of 128 per SM for each part: the register budget the compiler must
// meet and the grid's size (every block resident).  Each part is its own
// kernel, so the binning stages do not inherit the force loop's registers.
// Measured on 64 replicas (2.27M particles, FP32): part 0 at 10 blocks (48
// registers) and part 1 at 8 (64) take 1.99 ms per timestep against 2.05 at
// 6 and 6; in FP64, and for part 1 with a per-type table, those budgets
// spill, and both parts keep 6 (80 registers).
template <int PART, typename R, bool TYPED>
constexpr int p_blocks() {
  if constexpr (sizeof(R) == 8) return 6;
  else if constexpr (PART == 0) return 10;
  else return TYPED ? 6 : 8;
}
constexpr int kPMaxBlocksPerSM = 16;  // bound of every part's blocks (sizes the scan scratch)

template <typename R>
struct PArgs {
  using R4 = typename RT<R>::R4;
  // particle state: buffer cur in, buffer 1 - cur out
  R4* pos_c;
  R4* vel_c;
  const R* rc_c;
  const int32_t* id_c;
  R4* pos_o;
  R4* vel_o;
  R* rc_o;
  int32_t* id_o;
  R4* force;
  double* thermo;
  int64_t n;
  // binning
  int32_t* cell;
  int32_t* slot;
  int32_t* count;
  int32_t* start;
  int32_t* perm;
  int32_t* scan_blk;
  int64_t ncell;
  R l, il, lx, ilx;
  // replicas
  const RepGeom* geom;
  const uint16_t* rep_p;
  const uint16_t* rep_b;
  int nrep;
  // integration
  R hdt, dt;
  int drift, kick, recompute;
  // recomputation of interface, distances and cutoffs
  int64_t nbox;
  int32_t* box_count;
  int32_t* g;
  int32_t* g_tmp;
  uint8_t* s;
  uint8_t* iface;
  R* D0;
  R* D1;
  int32_t* flags;
  int32_t* thr;
  int32_t* hist;
  int w, fixed_thr, own_boxes, sweeps;
  R h, ih, r_grid, rc_min, rc_max, ramp;
  // forces
  ForceArgs<R> fa;
  const int2* tiles;
  int32_t ntiles;
  int32_t tile;          // particles per work item (a multiple of 32)
  R* w_i;
  int32_t* np_i;
  R* ke_i;
  // per-replica thermo
  const int64_t* chunk;
  int32_t nchunk;
  const int32_t* chunk0;
  double* tpart;
  // synchronisation
  uint32_t* sync;        // [0] arrivals, [1] generation, [2] abort, [3] force-queue head
  int32_t* status;
  int64_t budget_ns;     // longest barrier wait
  uint32_t phantom;      // blocks the barrier waits for beyond the grid (the self-test only)
  unsigned long long* pacc;  // nullable: [DCM_NSTAGES] nanoseconds per stage, [DCM_NSTAGES] runs, last stamp
};



// Stage timing of the persistent plan (dcm_batch_set_timing): block 0 reads
// the global timer whenever it leaves a barrier and charges the time since
// its previous reading to the stage that just ended (so a stage's time is
// the time until the grid's slowest block finished it).
__device__ __forceinline__ void stage_mark(unsigned long long* pacc, int stage) {
  if (pacc && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long t = global_ns();
    if (stage >= 0) {
      pacc[stage] += t - pacc[2 * DCM_NSTAGES];
      pacc[DCM_NSTAGES + stage] += 1;
    }
    pacc[2 * DCM_NSTAGES] = t;
  }
}

// Exclusive scan of v over the block (blockDim.x a multiple of 32, at most
// 1024); *total receives the block's sum.
__device__ __forceinline__ int block_scan_excl(int v, int* total) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) wsum[lane] = t;
  }
  __syncthreads();
  *total = wsum[nw - 1];
  return x - v + (wid > 0 ? wsum[wid - 1] : 0);
}

__device__ __forceinline__ int block_sum_int(int v) {
  int total;
  block_scan_excl(v, &total);
  return total;
}

// EW (part 1): the forces sum energy and virial and the thermo stages run
// (the last timestep of a call); otherwise the forces alone and the kick.
template <int PART, typename R, bool TYPED, bool X2, Accum M, bool EW>
__global__ void __launch_bounds__(kPBlock, (p_blocks<PART, R, TYPED>())) k_b_step_persistent(PArgs<R> a) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  const uint32_t expected = gridDim.x + a.phantom;
#define PSYNC()                                                    \
  do {                                                             \
    if (!grid_sync(a.sync, expected, a.budget_ns, a.status)) return; \
  } while (0)
#define PSTAGE(stage) stage_mark(a.pacc, stage)

  PSTAGE(-1);
  if constexpr (PART == 0) {
    // ---- clear the counters of this step
    for (int64_t c = gt; c < a.ncell; c += gs) a.count[c] = 0;
    if (a.recompute) {
      if (a.own_boxes)
        for (int64_t k = gt; k < a.nbox; k += gs) a.box_count[k] = 0;
      for (int64_t k = gt; k < (int64_t)a.nrep * kBatchHistBins; k += gs) a.hist[k] = 0;
      for (int64_t k = gt; k < a.sweeps + 2; k += gs) a.flags[k] = 0;
      for (int64_t r = gt; r < a.nrep; r += gs) b_thr_init((int)r, a.thr, a.fixed_thr);
    }
    if (gt == 0) a.sync[3] = 0;
    PSYNC();
    // ---- half kick, drift, cell counts
    for (int64_t i = gt; i < a.n; i += gs)
      b_kick_drift_count<R>(i, a.pos_c, a.vel_c, a.force, a.hdt, a.dt, a.l, a.il, a.lx, a.ilx, a.geom, a.rep_p,
                            a.cell, a.slot, a.count, a.drift);
    PSYNC();
    PSTAGE(DCM_STAGE_KICK_DRIFT);
    // ---- exclusive scan of the cell counts: each block owns one chunk
    const int64_t chunk = (a.ncell + gridDim.x - 1) / gridDim.x;
    const int64_t lo = min((int64_t)blockIdx.x * chunk, a.ncell), hi = min(lo + chunk, a.ncell);
    {
      int part = 0;
      for (int64_t c = lo + threadIdx.x; c < hi; c += blockDim.x) part += a.count[c];
      part = block_sum_int(part);
      if (threadIdx.x == 0) a.scan_blk[blockIdx.x] = part;
    }
    PSYNC();
    {
      int off = 0;
      for (int k = threadIdx.x; k < (int)blockIdx.x; k += blockDim.x) off += a.scan_blk[k];
      int run = block_sum_int(off);
      for (int64_t c0 = lo; c0 < hi; c0 += 4 * blockDim.x) {  // four cells per thread
        const int64_t c = c0 + 4 * threadIdx.x;
        int v[4], sum = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          v[q] = c + q < hi ? a.count[c + q] : 0;
          sum += v[q];
        }
        int tot;
        int ex = block_scan_excl(sum, &tot) + run;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (c + q < hi) a.start[c + q] = ex;
          ex += v[q];
        }
        run += tot;
      }
      if (hi == a.ncell && threadIdx.x == 0) a.start[a.ncell] = run;
    }
    PSYNC();
    // ---- stable counting sort: scatter, then order each cell by input index
    for (int64_t i = gt; i < a.n; i += gs) a.perm[a.start[a.cell[i]] + a.slot[i]] = (int32_t)i;
    PSYNC();
    for (int64_t c = gt; c < a.ncell; c += gs) b_sort_cell(a.start[c], a.start[c + 1], a.perm);
    PSYNC();
    for (int64_t k = gt; k < a.n; k += gs)
      b_gather<R>(k, a.perm, a.pos_c, a.pos_o, a.vel_c, a.vel_o, a.rc_c, a.rc_o, a.id_c, a.id_o);
    PSYNC();
    PSTAGE(DCM_STAGE_BIN);
    // ---- every K steps: interface, distances, cutoffs (Sections 2.1, 2.2)
    if (a.recompute) {
      const int32_t* counts = a.count;
      if (a.own_boxes) {
        for (int64_t i = gt; i < a.n; i += gs) b_box_count<R>(i, a.pos_o, a.h, a.ih, a.geom, a.rep_p, a.box_count);
        counts = a.box_count;
        PSYNC();
      }
      for (int64_t k = gt; k < a.nbox; k += gs) b_box_sum<0>(k, counts, a.g, a.geom, a.rep_b, a.w);
      PSYNC();
      for (int64_t k = gt; k < a.nbox; k += gs) b_box_sum<1>(k, a.g, a.g_tmp, a.geom, a.rep_b, a.w);
      PSYNC();
      for (int64_t k = gt; k < a.nbox; k += gs) b_box_sum<2>(k, a.g_tmp, a.g, a.geom, a.rep_b, a.w);
      PSYNC();
      if (a.fixed_thr < 0) {
        for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x; k0 < a.nbox; k0 += gs)
          b_minmax(k0 + threadIdx.x, a.g, a.nbox, a.rep_b, a.thr);
        PSYNC();
        for (int64_t k = gt; k < a.nbox; k += gs) b_value_hist(k, a.g, a.rep_b, a.thr, a.hist, a.status);
        PSYNC();
        for (int r = blockIdx.x; r < a.nrep; r += gridDim.x) b_two_means(r, a.hist, a.thr, 64);
        PSYNC();
      }
      for (int64_t k = gt; k < a.nbox; k += gs) b_segment(k, a.g, a.geom, a.rep_b, a.thr, a.s, a.iface);
      PSYNC();
      PSTAGE(DCM_STAGE_DETECT);
      for (int64_t k = gt; k < a.nbox; k += gs) b_dist_init<R>(k, a.s, a.iface, a.D0, a.D1);
      PSYNC();
      // Jacobi sweeps until one changes nothing (both buffers then agree) or
      // the even budget ends (the last iterate is then in D0)
      for (int it = 0; it < a.sweeps; ++it) {
        if (it > 0 && ((volatile int32_t*)a.flags)[it - 1] == 0) break;
        const R* Din = (it & 1) ? a.D1 : a.D0;
        R* Dout = (it & 1) ? a.D0 : a.D1;
        bool changed = false;
        for (int64_t k0 = (int64_t)blockIdx.x * blockDim.x; k0 < a.nbox; k0 += gs) {
          const int64_t k = k0 + threadIdx.x;
          if (k < a.nbox) changed |= b_dist_update<R, true>(k, Din, Dout, a.geom, a.rep_b, a.h, a.r_grid);
        }
        if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) a.flags[it] = 1;
        PSYNC();
      }
      if (gt == 0) {
        int first = -1;
        for (int k = 0; k < a.sweeps; ++k)
          if (a.flags[k] == 0) {
            first = k;
            break;
          }
        if (first < 0) raise_status(a.status, DCM_ERR_NOT_CONVERGED);
      }
      PSTAGE(DCM_STAGE_DISTANCE);
      for (int64_t i = gt; i < a.n; i += gs)
        b_cutoffs<R, false>(i, a.pos_o, a.D0, a.geom, a.rep_p, a.h, a.r_grid, a.rc_min, a.rc_max, a.ramp, a.rc_o);
      PSYNC();
      PSTAGE(DCM_STAGE_CUTOFFS);
    }
  } else {
    // ---- part 1: forces over the (replica, tile) queue (Section 2.4, Alg. 2.3).
    // Positions, cutoffs and cell starts were written by part 0, an earlier
    // launch, so they are read through the read-only path here.
    const int lane = threadIdx.x & 31;
    for (;;) {
      int t = 0;
      if (lane == 0) t = (int)atomicAdd(a.sync + 3, 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= a.ntiles) break;
      const int2 item = a.tiles[t];
      const int64_t end = min((int64_t)item.y + a.tile, a.geom[item.x].p1);
      for (int64_t i = (int64_t)item.y + lane; i < end; i += 32)
        b_force<R, TYPED, X2, M, true, EW>(i, a.pos_o, a.rc_o, a.start, a.fa, a.geom, a.rep_p, a.force, a.w_i,
                                           a.np_i);
    }
    PSYNC();
    PSTAGE(DCM_STAGE_FORCES);
    // ---- second half kick, kinetic energy, per-replica thermo
    for (int64_t i = gt; i < a.n; i += gs)
      b_kick<R>(i, a.vel_o, a.kick ? a.force : nullptr, a.hdt, EW ? a.ke_i : nullptr);
    if constexpr (EW) {
      PSYNC();
      for (int c = blockIdx.x; c < a.nchunk; c += gridDim.x)
        b_thermo_chunk<R>(c, a.chunk, a.nchunk, a.force, a.w_i, a.ke_i, a.np_i, a.tpart);
      PSYNC();
      const int64_t warp = gt >> 5, nwarp = gs >> 5;
      for (int64_t r = warp; r < a.nrep; r += nwarp) b_thermo_sum((int)r, a.chunk0, a.nchunk, a.tpart, a.thermo);
    }
    // the kick's time: up to the last barrier (the thermo sums of the last
    // warps are not waited for)
    PSTAGE(DCM_STAGE_KICK);
  }
#undef PSTAGE
#undef PSYNC
}

// The barrier alone, for the self-test of its bounded wait.
__global__ void __launch_bounds__(kPBlock) k_b_wait_selftest(uint32_t* sync, uint32_t expected, int64_t budget_ns,
                                                             int32_t* status) {
  grid_sync(sync, expected, budget_ns, status);
}

namespace {

// One cooperative launch of part PART over as many blocks as are resident
// (at most the part's cap per SM); the barrier words start cleared.
template <int PART, typename R, bool TYPED, bool X2, Accum M, bool EW>
int launch_part(dcm_batch* b, const PArgs<R>& a, cudaStream_t st) {
  auto kern = k_b_step_persistent<PART, R, TYPED, X2, M, EW>;
  int per_sm = 0, sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPBlock, 0) != cudaSuccess || per_sm < 1)
    return set_error(&b->base, DCM_ERR_CUDA, "persistent step: occupancy query failed");
  const int grid = std::min(per_sm, p_blocks<PART, R, TYPED>()) * sms;
  if (grid > b->pgrid) return set_error(&b->base, DCM_ERR_CAPACITY, "persistent grid %d exceeds its scratch", grid);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaMemsetAsync(b->sync, 0, 4 * sizeof(uint32_t), st) != cudaSuccess)
    return set_error(&b->base, DCM_ERR_CUDA, "persistent step: memset failed");
  ++b->base.launches;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return set_error(&b->base, DCM_ERR_CUDA, "persistent step: %s", cudaGetErrorString(e));
  return DCM_OK;
}

// part 0 (binning, recomputation), then part 1 (forces, kick, thermo); the
// scalar loop (X2 false) always sums energy and virial
template <typename R, bool TYPED, bool X2, Accum M>
int launch_persistent(dcm_batch* b, const PArgs<R>& a, cudaStream_t st, bool energies) {
  int r = launch_part<0, R, TYPED, X2, M, true>(b, a, st);
  if (r != DCM_OK) return r;
  if constexpr (X2) {
    if (!energies) return launch_part<1, R, TYPED, X2, M, false>(b, a, st);
  }
  return launch_part<1, R, TYPED, X2, M, true>(b, a, st);
}

template <typename R>
int dispatch_persistent(dcm_batch* b, const PArgs<R>& a, cudaStream_t st, bool energies) {
  const LJTable t = lj_table(b->p);
  const bool typed = lj_general(t);
  if constexpr (sizeof(R) == 8) {
    return typed ? launch_persistent<R, true, false, Accum::kPlain>(b, a, st, energies)
                 : launch_persistent<R, false, false, Accum::kPlain>(b, a, st, energies);
  } else {
    const bool x2 = !(typed && t.ntypes > 2);
    auto go = [&](auto tag) {
      constexpr Accum M = decltype(tag)::value;
      if (!x2) return launch_persistent<R, true, false, M>(b, a, st, energies);
      return typed ? launch_persistent<R, true, true, M>(b, a, st, energies)
                   : launch_persistent<R, false, true, M>(b, a, st, energies);
    };
    const int acc = batch_accumulation(b);
    if (acc == DCM_ACC_FP32) return go(AccumTag<Accum::kPlain>{});
    if (acc == DCM_ACC_PLANE_FP64) return go(AccumTag<Accum::kPlaneF64>{});
    return go(AccumTag<Accum::kPlaneKahan>{});
  }
}

}  // namespace

// The (replica, first particle) work items of `tile` particles each; no item
// spans two replicas.
static int build_tiles(dcm_batch* b, int tile) {
  std::vector<int2> tiles;
  for (int r = 0; r < b->R; ++r)
    for (int64_t i = b->geom_h[(size_t)r].p0; i < b->geom_h[(size_t)r].p1; i += tile)
      tiles.push_back(make_int2(r, (int)i));
  int2* dev = nullptr;
  if (cudaMalloc((void**)&dev, sizeof(int2) * std::max<size_t>(tiles.size(), 1)) != cudaSuccess) return DCM_ERR_NOMEM;
  if (!tiles.empty() && cudaMemcpy(dev, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dev);
    return DCM_ERR_CUDA;
  }
  if (b->tiles) cudaFree(b->tiles);
  b->tiles = dev;
  b->ntiles = (int32_t)tiles.size();
  b->tile = tile;
  return DCM_OK;
}

int b_persistent_setup(dcm_batch* b) {
  if (b->tiles) return DCM_OK;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DCM_ERR_CUDA;
  b->pgrid = sms * kPMaxBlocksPerSM;
  if (cudaMalloc((void**)&b->sync, 4 * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc((void**)&b->scan_blk, sizeof(int32_t) * (size_t)b->pgrid) != cudaSuccess ||
      cudaMalloc((void**)&b->pacc, sizeof(unsigned long long) * (2 * DCM_NSTAGES + 1)) != cudaSuccess)
    return DCM_ERR_NOMEM;
  if (cudaMemset(b->sync, 0, 4 * sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(b->pacc, 0, sizeof(unsigned long long) * (2 * DCM_NSTAGES + 1)) != cudaSuccess)
    return DCM_ERR_CUDA;
  return build_tiles(b, kQueueTile);
}

int b_persistent_set_tile(dcm_batch* b, int tile) {
  if (tile < 32 || tile > 4096 || tile % 32) return DCM_ERR_INVALID_ARG;
  return build_tiles(b, tile);
}

template <typename R>
int b_persistent_step(dcm_batch* b, dcm_state* s, R hdt, R dt, bool drift, bool recompute, bool kick,
                      bool energies, cudaStream_t st) {
  using R4 = typename RT<R>::R4;
  dcm_ctx* ctx = &b->base;
  const dcm_params& p = b->p;
  const int c = s->cur, o = 1 - c;
  const bool ids = s->id[c] && s->id[o];
  PArgs<R> a;
  memset(&a, 0, sizeof(a));
  a.pos_c = (R4*)s->pos[c];
  a.vel_c = (R4*)s->vel[c];
  a.rc_c = (const R*)s->rc[c];
  a.id_c = ids ? s->id[c] : nullptr;
  a.pos_o = (R4*)s->pos[o];
  a.vel_o = (R4*)s->vel[o];
  a.rc_o = (R*)s->rc[o];
  a.id_o = ids ? s->id[o] : nullptr;
  a.force = (R4*)s->force;
  a.thermo = s->thermo;
  a.n = b->ntot;
  a.cell = ctx->cell;
  a.slot = ctx->slot;
  a.count = ctx->cell_count;
  a.start = ctx->cell_start;
  a.perm = ctx->perm;
  a.scan_blk = b->scan_blk;
  a.ncell = b->ncell_tot;
  a.l = (R)p.l;
  a.il = (R)(1.0 / p.l);
  a.lx = (R)p.lx;
  a.ilx = (R)(1.0 / p.lx);
  a.geom = b->geom;
  a.rep_p = b->rep_of_particle;
  a.rep_b = b->rep_of_box;
  a.nrep = b->R;
  a.hdt = hdt;
  a.dt = dt;
  a.drift = drift;
  a.kick = kick;
  a.recompute = recompute;
  a.nbox = b->nbox_tot;
  a.box_count = ctx->box_count;
  a.g = ctx->g;
  a.g_tmp = ctx->g_tmp;
  a.s = ctx->s;
  a.iface = ctx->iface;
  a.D0 = (R*)ctx->D[0];
  a.D1 = (R*)ctx->D[1];
  a.flags = ctx->flags;
  a.thr = b->thr;
  a.hist = b->hist;
  a.w = p.smooth_w;
  a.fixed_thr = p.threshold;
  a.own_boxes = (p.h != p.l || p.lx != p.l) ? 1 : 0;
  a.sweeps = p.iter_max + (p.iter_max & 1);  // the sweep loop leaves once a sweep changes nothing
  a.h = (R)p.h;
  a.ih = (R)(1.0 / p.h);
  a.r_grid = (R)p.r_grid;
  a.rc_min = (R)p.rc_min;
  a.rc_max = (R)p.rc_max;
  a.ramp = (R)p.ramp;
  a.fa = batch_force_args<R>(b);
  a.tiles = b->tiles;
  a.ntiles = b->ntiles;
  a.tile = b->tile;
  a.w_i = (R*)b->w_i;
  a.np_i = b->np_i;
  a.ke_i = (R*)b->ke_i;
  a.chunk = b->chunk;
  a.nchunk = b->nchunk;
  a.chunk0 = b->chunk0;
  a.tpart = b->tpart;
  a.sync = b->sync;
  a.status = ctx->status;
  a.budget_ns = b->wait_budget;
  a.phantom = 0;
  a.pacc = b->base.timing ? b->pacc : nullptr;
  if (b->ntot == 0) return DCM_OK;
  int r = dispatch_persistent<R>(b, a, st, energies);
  return r ? r : check_launch(ctx, "persistent step");
}

template int b_persistent_step<float>(dcm_batch*, dcm_state*, float, float, bool, bool, bool, bool, cudaStream_t);
template int b_persistent_step<double>(dcm_batch*, dcm_state*, double, double, bool, bool, bool, bool, cudaStream_t);

int b_persistent_wait_selftest(dcm_batch* b, int32_t phantom, int64_t budget_ns, cudaStream_t st) {
  int r = b_persistent_setup(b);
  if (r) return r;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_wait_selftest, kPBlock, 0) != cudaSuccess)
    return DCM_ERR_CUDA;
  const int grid = std::min(per_sm, kPMaxBlocksPerSM) * sms;
  if (cudaMemsetAsync(b->sync, 0, 4 * sizeof(uint32_t), st) != cudaSuccess) return DCM_ERR_CUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kPBlock);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++b->base.launches;
  if (cudaLaunchKernelEx(&cfg, k_b_wait_selftest, b->sync, (uint32_t)grid + (uint32_t)std::max(phantom, 0),
                         budget_ns, b->base.status) != cudaSuccess)
    return DCM_ERR_CUDA;
  return dcm_status(&b->base, (dcm_stream_t)st);
}

}  // namespace dcm
