// Per-particle cutoffs (Section 2.2): particle-interface distance by trilinear
// interpolation of the box distances, then the cutoff rule.
//
// The interpolation offset t = (x - (k + 1/2) h) / h is formed from an exact
// subtraction (k is the exact floor and (k + 1/2) h is representable), so the
// weights carry one rounding even at the far end of a large box.
#include "dcm_internal.cuh"

namespace dcm {

template <typename R>
__device__ __forceinline__ void centre_coord(R x, R h, R inv_h, int& k, R& t) {
  R q = floor(x * inv_h - (R)0.5);
  k = (int)q;
  if (((R)k + (R)0.5) * h > x)
    --k;
  else if (((R)k + (R)1.5) * h <= x)
    ++k;
  t = (x - ((R)k + (R)0.5) * h) / h;
}

template <typename R>
__global__ void k_cutoffs(int64_t n, const typename RT<R>::R4* __restrict__ pos, const R* __restrict__ D, int nx,
                          int ny, int nz, R h, R inv_h, R r_grid, R rc_min, R rc_max, R ramp, R* __restrict__ rc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto p = ldg4(pos + i);
  int kx, ky, kz;
  R tx, ty, tz;
  centre_coord<R>(p.x, h, inv_h, kx, tx);
  centre_coord<R>(p.y, h, inv_h, ky, ty);
  centre_coord<R>(p.z, h, inv_h, kz, tz);
  // periodic wrap (a true modulo, so positions outside the box stay in range)
  auto wrapk = [](int k, int n) { k %= n; return k < 0 ? k + n : k; };
  int x0 = wrapk(kx, nx), x1 = wrapk(kx + 1, nx);
  int y0 = wrapk(ky, ny), y1 = wrapk(ky + 1, ny);
  int z0 = wrapk(kz, nz), z1 = wrapk(kz + 1, nz);
  auto at = [&](int x, int y, int z) {
    R v = D[x + (int64_t)nx * (y + (int64_t)ny * z)];
    return v < r_grid ? v : r_grid;
  };
  // nested linear interpolation: a + t (b - a)
  auto lerp = [](R a, R b, R t) { return fma(t, b - a, a); };
  R c00 = lerp(at(x0, y0, z0), at(x1, y0, z0), tx);
  R c10 = lerp(at(x0, y1, z0), at(x1, y1, z0), tx);
  R c01 = lerp(at(x0, y0, z1), at(x1, y0, z1), tx);
  R c11 = lerp(at(x0, y1, z1), at(x1, y1, z1), tx);
  R c0 = lerp(c00, c10, ty), c1 = lerp(c01, c11, ty);
  R delta = lerp(c0, c1, tz);
  R r;
  if (ramp > (R)0) {
    r = rc_max - (rc_max - rc_min) * delta / ramp;
    r = r < rc_min ? rc_min : (r > rc_max ? rc_max : r);
  } else {
    r = delta > (R)0 ? rc_min : rc_max;
  }
  rc[i] = r;
}

template <typename R>
int assign_cutoffs(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* D, R* rc, cudaStream_t st) {
  if (n > 0) {
    const dcm_params& p = ctx->p;
    DCM_LAUNCH(ctx, k_cutoffs<R>, (unsigned)((n + 255) / 256), 256, 0, st, 
        n, pos, D, (int)ctx->nh[0], (int)ctx->nh[1], (int)ctx->nh[2], (R)p.h, (R)(1.0 / p.h), (R)p.r_grid,
        (R)p.rc_min, (R)p.rc_max, (R)p.ramp, rc);
  }
  return check_launch(ctx, "assign_cutoffs");
}

template int assign_cutoffs<float>(dcm_ctx*, int64_t, const float4*, const float*, float*, cudaStream_t);
template int assign_cutoffs<double>(dcm_ctx*, int64_t, const dvec4*, const double*, double*, cudaStream_t);

}  // namespace dcm
