// Box-interface distances (Section 2.2, Algorithm 2.1): cutoff-based fast
// sweeping on the density-box grid.
//
// Algorithm 2.1 processes a queue of boxes breadth-first and keeps going
// until the largest change of a pass is below epsilon; its result is the
// fixed point of the local fast-sweeping update restricted to distances
// <= r_grid, whatever the visiting order.  On the GPU the same fixed point is
// reached by Jacobi sweeps: every box of the high-density phase re-solves the
// Godunov update from the previous iterate (double buffered, so the result is
// deterministic), and a per-sweep device flag records whether any box
// changed; a sweep that finds its predecessor's flag clear exits at once, so
// a fixed budget of launches costs little once converged.  The MPI_Allreduce
// of the paper's version becomes that flag.
#include <algorithm>

#include "dcm_internal.cuh"

namespace dcm {

template <typename R>
__global__ void k_dist_init(const uint8_t* __restrict__ s, const uint8_t* __restrict__ iface, int64_t nbox,
                            R* __restrict__ D0, R* __restrict__ D1) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  R v = (!s[b] || iface[b]) ? (R)0 : RT<R>::inf();
  D0[b] = v;
  D1[b] = v;
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

// One Jacobi sweep.  Grid-stride over (row, chunk) work items with a grid of
// a few waves, so a sweep after convergence costs one short wave of blocks
// that read the flag and leave.
template <typename R>
__global__ void k_dist_sweep(const R* __restrict__ Din, R* __restrict__ Dout, int nx, int ny, int nz, R h, R r_grid,
                             int32_t* __restrict__ flags, int it) {
  if (it > 0 && flags[it - 1] == 0) return;  // the previous sweep changed nothing: converged
  const int chunks = (nx + blockDim.x - 1) / blockDim.x;
  const int64_t items = (int64_t)ny * nz * chunks;
  bool changed = false;
  for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
    int yz = (int)(w / chunks);
    int x = (int)(w - (int64_t)yz * chunks) * blockDim.x + threadIdx.x;
    if (x >= nx) continue;
    int y = yz % ny, z = yz / ny;
    int64_t b = x + (int64_t)nx * yz;
    R cur = Din[b];
    if (cur == (R)0) continue;  // interface / low-density boxes are fixed at 0 in both buffers
    int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    int64_t row = (int64_t)nx * (y + (int64_t)ny * z);
    R a0 = fmin(Din[row + xm], Din[row + xp]);
    R a1 = fmin(Din[x + nx * (ym + (int64_t)ny * z)], Din[x + nx * (yp + (int64_t)ny * z)]);
    R a2 = fmin(Din[x + nx * (y + (int64_t)ny * zm)], Din[x + nx * (y + (int64_t)ny * zp)]);
    R d = godunov3<R>(a0, a1, a2, h);
    R out = cur;
    if (d < cur && d <= r_grid) {
      out = d;
      changed = true;
    }
    Dout[b] = out;
  }
  if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) flags[it] = 1;
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
  unsigned nb = (unsigned)((nbox + 255) / 256);
  int64_t items = (int64_t)ny * nz * ((nx + 127) / 128);
  unsigned sg = (unsigned)std::min<int64_t>(items, 152 * 16);
  int iter_max = ctx->p.iter_max;
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->flags, 0, sizeof(int32_t) * (size_t)(iter_max + 2), st));
  DCM_LAUNCH(ctx, k_dist_init<R>, nb, 256, 0, st, s, iface, nbox, buf[0], buf[1]);
  int done = 0;
  if (host_check) {
    // chunks of 8 sweeps, then look at the last flag of the chunk on the host
    const int chunk = 8;
    bool converged = false;
    while (done < iter_max && !converged) {
      int m = std::min(chunk, iter_max - done);
      for (int k = 0; k < m; ++k, ++done)
        DCM_LAUNCH(ctx, k_dist_sweep<R>, sg, 128, 0, st, buf[done & 1], buf[(done + 1) & 1], nx, ny, nz, h, rg, ctx->flags, done);
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
    // fixed even budget (result ends in buf[0] = D).  Along a front the
    // Godunov update can add arbitrarily little per box, so the sweep count is
    // not bounded by r_grid / h; 8 r_grid / h + 8 leaves a wide margin over
    // what wavy slab interfaces need (about 5 r_grid / h), and sweeps after
    // convergence exit at once.
    int budget = (int)std::ceil(8.0 * ctx->p.r_grid / ctx->p.h) + 8;
    budget = std::min(budget + (budget & 1), iter_max + (iter_max & 1));
    for (; done < budget; ++done)
      DCM_LAUNCH(ctx, k_dist_sweep<R>, sg, 128, 0, st, buf[done & 1], buf[(done + 1) & 1], nx, ny, nz, h, rg, ctx->flags, done);
    DCM_LAUNCH(ctx, k_dist_finish, 1, 1, 0, st, ctx->flags, done, iters, ctx->status);
  }
  return check_launch(ctx, "distance_sweeps");
}

template int distance_sweeps<float>(dcm_ctx*, const uint8_t*, const uint8_t*, float*, int32_t*, bool, cudaStream_t);
template int distance_sweeps<double>(dcm_ctx*, const uint8_t*, const uint8_t*, double*, int32_t*, bool,
                                     cudaStream_t);

}  // namespace dcm
