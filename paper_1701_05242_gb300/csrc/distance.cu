// Box-interface distances (Section 2.2, Algorithm 2.1): cutoff-based fast
// sweeping on the density-box grid.
//
// Algorithm 2.1 processes a queue of boxes breadth-first and keeps going
// until the largest change of a pass is below epsilon; its result is the
// fixed point of the local fast-sweeping update restricted to distances
// <= r_grid, whatever the visiting order.  On the GPU the same fixed point is
// reached by Jacobi sweeps (double buffered, so the result is deterministic):
// sweep 0 re-solves every box of the high-density phase; every later sweep
// re-solves only the boxes of its queue — the boxes that changed in the
// previous sweep and their six neighbours — which are exactly the boxes
// whose update can differ from the previous sweep's, so the iterates are
// those of full Jacobi sweeps while the work follows the moving front (the
// paper's queue Q); the MPI_Allreduce of the paper's version becomes the
// queue length in device memory.  dcm_distance launches one kernel per sweep
// and checks convergence on the host every eight sweeps; the timestep runs
// every sweep in one cooperative launch with a grid barrier between sweeps
// (no host wait), until a sweep changes nothing or iter_max sweeps have run.
#include <algorithm>

#include "dcm_internal.cuh"
#include "grid_sync.cuh"

namespace dcm {

template <typename R>
__global__ void k_dist_init(const uint8_t* __restrict__ s, const uint8_t* __restrict__ iface, int64_t nbox,
                            R* __restrict__ D0, R* __restrict__ D1, uint8_t* __restrict__ fixed0,
                            int32_t* __restrict__ stamp) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  bool z = !s[b] || iface[b];
  R v = z ? (R)0 : RT<R>::inf();
  D0[b] = v;
  D1[b] = v;
  fixed0[b] = (uint8_t)z;
  stamp[b] = -1;
}

// Godunov upwind update of |grad d| = 1 with spacing h from the three axis
// minima a (any order).  Returns +inf if all are +inf.
template <typename R>
__device__ __forceinline__ R godunov3(R a0, R a1, R a2, R h) {
  // sort ascending
  R t;
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  R d = a0 + h;
  if (d > a1) {
    R df = a0 - a1;
    d = (R)0.5 * (a0 + a1 + sqrt((R)2 * h * h - df * df));
    if (d > a2) {
      R sa = a0 + a1 + a2;
      R sq = a0 * a0 + a1 * a1 + a2 * a2;
      R disc = sa * sa - (R)3 * (sq - h * h);
      d = (sa + sqrt(disc > (R)0 ? disc : (R)0)) / (R)3;
    }
  }
  return d;
}

// Queue the high-density boxes among b and its six neighbours for sweep it+1
// (each box once: stamp holds the last sweep a box was queued for).
__device__ __forceinline__ void dist_push(int64_t b, int x, int y, int z, int nx, int ny, int nz,
                                          const uint8_t* __restrict__ fixed0, int32_t* __restrict__ stamp,
                                          int32_t* __restrict__ qout, int32_t* __restrict__ qlen, int it) {
  const int64_t nxy = (int64_t)nx * ny;
  int64_t nb[7] = {b,
                   x == 0 ? b + nx - 1 : b - 1,
                   x == nx - 1 ? b - x : b + 1,
                   y == 0 ? b + (int64_t)(ny - 1) * nx : b - nx,
                   y == ny - 1 ? b - (int64_t)y * nx : b + nx,
                   z == 0 ? b + (int64_t)(nz - 1) * nxy : b - nxy,
                   z == nz - 1 ? b - (int64_t)z * nxy : b + nxy};
  for (int k = 0; k < 7; ++k) {
    int64_t q = nb[k];
    if (fixed0[q]) continue;
    if (atomicExch(stamp + q, it + 1) != it + 1) qout[atomicAdd(qlen + it + 1, 1)] = (int32_t)q;
  }
}

// Loads of the iterates: COH through L2 (__ldcg), for the cooperative sweep
// kernel, whose blocks read what other blocks wrote earlier in the same
// launch (behind a grid barrier); ordinary loads otherwise.
template <typename R, bool COH>
__device__ __forceinline__ R dld(const R* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// Update of one box from the previous iterate; true if it changed.
template <typename R, bool COH = false>
__device__ __forceinline__ bool dist_update(const R* Din, R* Dout, int64_t b, int x, int y, int z, int nx, int ny,
                                            int nz, R h, R r_grid) {
  R cur = dld<R, COH>(Din + b);
  int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  int64_t row = (int64_t)nx * (y + (int64_t)ny * z);
  R a0 = fmin(dld<R, COH>(Din + row + xm), dld<R, COH>(Din + row + xp));
  R a1 = fmin(dld<R, COH>(Din + x + nx * (ym + (int64_t)ny * z)), dld<R, COH>(Din + x + nx * (yp + (int64_t)ny * z)));
  R a2 = fmin(dld<R, COH>(Din + x + nx * (y + (int64_t)ny * zm)), dld<R, COH>(Din + x + nx * (y + (int64_t)ny * zp)));
  R d = godunov3<R>(a0, a1, a2, h);
  bool ch = d < cur && d <= r_grid;
  Dout[b] = ch ? d : cur;
  return ch;
}

// Sweep 0 over the whole grid.  Grid-stride over (row, chunk) work items.
template <typename R>
__global__ void k_dist_sweep0(const R* __restrict__ Din, R* __restrict__ Dout, int nx, int ny, int nz, R h, R r_grid,
                              const uint8_t* __restrict__ fixed0, int32_t* __restrict__ stamp,
                              int32_t* __restrict__ qout, int32_t* __restrict__ qlen, int32_t* __restrict__ flags) {
  const int chunks = (nx + blockDim.x - 1) / blockDim.x;
  const int64_t items = (int64_t)ny * nz * chunks;
  bool changed = false;
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    int yz = (int)(w / chunks);
    int x = (int)(w - (int64_t)yz * chunks) * blockDim.x + threadIdx.x;
    if (x >= nx) continue;
    int y = yz % ny, z = yz / ny;
    int64_t b = x + (int64_t)nx * yz;
    if (fixed0[b]) continue;  // interface / low-density boxes are fixed at 0 in both buffers
    if (dist_update<R>(Din, Dout, b, x, y, z, nx, ny, nz, h, r_grid)) {
      changed = true;
      dist_push(b, x, y, z, nx, ny, nz, fixed0, stamp, qout, qlen, 0);
    }
  }
  if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) flags[0] = 1;
}

// Sweep it >= 1 over its queue (grid-stride; an empty queue means converged).
template <typename R>
__global__ void k_dist_sweep_queue(const R* __restrict__ Din, R* __restrict__ Dout, int nx, int ny, int nz, R h,
                                   R r_grid, const uint8_t* __restrict__ fixed0, int32_t* __restrict__ stamp,
                                   const int32_t* __restrict__ qin, int32_t* __restrict__ qout,
                                   int32_t* __restrict__ qlen, int32_t* __restrict__ flags, int it) {
  const int32_t n = qlen[it];
  bool changed = false;
  const int64_t nxy = (int64_t)nx * ny;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = qin[k];
    int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / nxy);
    if (dist_update<R>(Din, Dout, b, x, y, z, nx, ny, nz, h, r_grid)) {
      changed = true;
      dist_push(b, x, y, z, nx, ny, nz, fixed0, stamp, qout, qlen, it);
    }
  }
  if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) flags[it] = 1;
}

// All sweeps in one cooperative launch (every block resident): sweep 0 over
// the whole grid, then the queue sweeps, a bounded grid barrier after each,
// until a sweep changes nothing or `budget` sweeps have run.  The same
// iterates as one launch per sweep (bit for bit); the loop needs no host
// check and launches nothing per sweep.  A barrier wait that runs past
// budget_ns records DCM_ERR_TIMEOUT and ends the launch.
template <typename R>
__global__ void __launch_bounds__(256) k_dist_coop(R* D0, R* D1, int nx, int ny, int nz, R h, R r_grid,
                                                   const uint8_t* __restrict__ fixed0, int32_t* stamp, int32_t* q0,
                                                   int32_t* q1, int32_t* qlen, int32_t* flags, int budget,
                                                   uint32_t* sync, int64_t budget_ns, int32_t* status) {
  const unsigned full = 0xffffffffu;
  const uint32_t expected = gridDim.x;
  const int64_t nxy = (int64_t)nx * ny;
  {
    const int chunks = (nx + blockDim.x - 1) / blockDim.x;
    const int64_t items = (int64_t)ny * nz * chunks;
    bool changed = false;
    for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
      const int yz = (int)(w / chunks);
      const int x = (int)(w - (int64_t)yz * chunks) * blockDim.x + threadIdx.x;
      if (x >= nx) continue;
      const int y = yz % ny, z = yz / ny;
      const int64_t b = x + (int64_t)nx * yz;
      if (fixed0[b]) continue;
      if (dist_update<R, true>(D0, D1, b, x, y, z, nx, ny, nz, h, r_grid)) {
        changed = true;
        dist_push(b, x, y, z, nx, ny, nz, fixed0, stamp, q1, qlen, 0);
      }
    }
    if (__any_sync(full, changed) && (threadIdx.x & 31) == 0) flags[0] = 1;
  }
  if (!grid_sync(sync, expected, budget_ns, status)) return;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
  for (int it = 1; it < budget; ++it) {
    if (((volatile int32_t*)flags)[it - 1] == 0) break;  // the previous sweep changed nothing
    const R* Din = (it & 1) ? D1 : D0;
    R* Dout = (it & 1) ? D0 : D1;
    const int32_t* qin = (it & 1) ? q1 : q0;
    int32_t* qout = (it & 1) ? q0 : q1;
    const int32_t n = ((volatile int32_t*)qlen)[it];
    bool changed = false;
    for (int64_t k = gt; k < n; k += gs) {
      const int64_t b = __ldcg(qin + k);
      const int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / nxy);
      if (dist_update<R, true>(Din, Dout, b, x, y, z, nx, ny, nz, h, r_grid)) {
        changed = true;
        dist_push(b, x, y, z, nx, ny, nz, fixed0, stamp, qout, qlen, it);
      }
    }
    if (__any_sync(full, changed) && (threadIdx.x & 31) == 0) flags[it] = 1;
    if (!grid_sync(sync, expected, budget_ns, status)) return;
  }
}

// iters = 1 + index of the first sweep that changed nothing (or -1), and a
// device status if the budget ran out.
__global__ void k_dist_finish(const int32_t* flags, int sweeps, int32_t* iters, int32_t* status) {
  int first = -1;
  for (int k = 0; k < sweeps; ++k)
    if (flags[k] == 0) {
      first = k;
      break;
    }
  if (iters) *iters = first >= 0 ? first + 1 : -1;
  if (first < 0) raise_status(status, DCM_ERR_NOT_CONVERGED);
}

template <typename R>
int distance_sweeps(dcm_ctx* ctx, const uint8_t* s, const uint8_t* iface, R* D, int32_t* iters, bool host_check,
                    cudaStream_t st) {
  int nx = (int)ctx->nh[0], ny = (int)ctx->nh[1], nz = (int)ctx->nh[2];
  int64_t nbox = ctx->nbox;
  R h = (R)ctx->p.h, rg = (R)ctx->p.r_grid;
  R* buf[2] = {D, (R*)ctx->D[1]};
  int32_t* q[2] = {ctx->dq[0], ctx->dq[1]};
  unsigned nb = (unsigned)((nbox + 255) / 256);
  int64_t items = (int64_t)ny * nz * ((nx + 127) / 128);
  unsigned sg = (unsigned)std::min<int64_t>(items, 152 * 16);
  const unsigned qg = 152 * 8;  // queue sweeps: grid-stride over the queue length read on the device
  int iter_max = ctx->p.iter_max;
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->flags, 0, sizeof(int32_t) * (size_t)(iter_max + 2), st));
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dqlen, 0, sizeof(int32_t) * (size_t)(iter_max + 2), st));
  DCM_LAUNCH(ctx, k_dist_init<R>, nb, 256, 0, st, s, iface, nbox, buf[0], buf[1], ctx->dfixed, ctx->dstamp);
  auto sweep = [&](int it) -> int {
    if (it == 0)
      DCM_LAUNCH(ctx, k_dist_sweep0<R>, sg, 128, 0, st, buf[0], buf[1], nx, ny, nz, h, rg, ctx->dfixed, ctx->dstamp,
                 q[1], ctx->dqlen, ctx->flags);
    else
      DCM_LAUNCH(ctx, k_dist_sweep_queue<R>, qg, 256, 0, st, buf[it & 1], buf[(it + 1) & 1], nx, ny, nz, h, rg,
                 ctx->dfixed, ctx->dstamp, q[it & 1], q[(it + 1) & 1], ctx->dqlen, ctx->flags, it);
    return DCM_OK;
  };
  int done = 0;
  if (host_check) {
    // chunks of 8 sweeps, then look at the last flag of the chunk on the host
    const int chunk = 8;
    bool converged = false;
    while (done < iter_max && !converged) {
      int m = std::min(chunk, iter_max - done);
      for (int k = 0; k < m; ++k, ++done) sweep(done);
      DCM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->host_status, ctx->flags + done - 1, sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, st));
      DCM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
      converged = ctx->host_status[0] == 0;
    }
    DCM_LAUNCH(ctx, k_dist_finish, 1, 1, 0, st, ctx->flags, done, iters, ctx->status);
    if (!converged) {
      if (done & 1) DCM_CUDA_TRY(ctx, cudaMemcpyAsync(D, buf[1], sizeof(R) * nbox, cudaMemcpyDeviceToDevice, st));
      check_launch(ctx, "distance_sweeps");
      return set_error(ctx, DCM_ERR_NOT_CONVERGED, "fast sweeping did not converge in %d sweeps", iter_max);
    }
  } else {
    // every sweep in one cooperative launch, until one changes nothing or
    // the even budget iter_max (rounded up) runs out (the last iterate then
    // in buf[0] = D); no host check
    const int budget = iter_max + (iter_max & 1);
    auto kern = k_dist_coop<R>;
    int per_sm = 0, sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess || per_sm < 1)
      return set_error(ctx, DCM_ERR_CUDA, "distance sweeps: occupancy query failed");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(std::min(per_sm, 4) * sms));
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, buf[0], buf[1], nx, ny, nz, h, rg, (const uint8_t*)ctx->dfixed,
                                       ctx->dstamp, q[0], q[1], ctx->dqlen, ctx->flags, budget, ctx->coop_sync,
                                       (int64_t)2000000000, ctx->status);
    if (e != cudaSuccess) return set_error(ctx, DCM_ERR_CUDA, "distance sweeps: %s", cudaGetErrorString(e));
    done = budget;
    DCM_LAUNCH(ctx, k_dist_finish, 1, 1, 0, st, ctx->flags, done, iters, ctx->status);
  }
  return check_launch(ctx, "distance_sweeps");
}

template int distance_sweeps<float>(dcm_ctx*, const uint8_t*, const uint8_t*, float*, int32_t*, bool, cudaStream_t);
template int distance_sweeps<double>(dcm_ctx*, const uint8_t*, const uint8_t*, double*, int32_t*, bool,
                                     cudaStream_t);

}  // namespace dcm
