// Regularised two-phase segmentation of the box counts (Section 2.1: the
// piecewise constant Mumford-Shah functional for two-phase segmentation,
// refs. [1, 18]), selected by params.segmentation = 1.
//
// The functional of a binary volume s with phase values c0, c1 is
//   E(s) = sum_b [ s_b (g_b - c1)^2 + (1 - s_b) (g_b - c0)^2 ] + nu sum_faces |s_b - s_b'|
// on the periodic grid of box counts g.  Starting from the threshold
// segmentation, each outer iteration sets c0, c1 to the means of g over the
// two phases (exact integer sums), then minimises the convex relaxation
//   min over u in [0,1]: sum_b w_b u_b + nu sum_faces |u_b - u_b'|,
//   w_b = (g_b - c1)^2 - (g_b - c0)^2,
// by the primal-dual iteration of Chambolle and Pock (one dual value per
// face, a stencil on the grid), and thresholds u at 1/2.  The loop stops
// after params.ms_outer iterations or when s no longer changes; the later
// launches of a finished loop exit at once (a device flag per iteration), so
// the host never waits.  Additions and products are rounded one by one
// (no fused multiply-add), in the order of the plain definition, so the FP64
// form reproduces an FP64 evaluation of the same steps.
#include "dcm_internal.cuh"

namespace dcm {

namespace {

constexpr double kMsTau = 0.28, kMsSigma = 0.28;  // tau sigma ||D||^2 < 1 with ||D||^2 <= 12

__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }

// Whether outer iteration o still runs: the earlier ones changed s, and both
// phases were present when it started (flags[0] is the stop mark).
__device__ __forceinline__ bool ms_active(const int32_t* flags, int o) {
  return flags[0] == 0 && (o == 0 || flags[o] != 0);
}

// Integer sums of the counts over the two phases: sums = {n0, S0, n1, S1}.
__global__ void k_ms_sums(const int32_t* __restrict__ g, const uint8_t* __restrict__ s, int64_t nbox,
                          unsigned long long* sums, const int32_t* flags, int o) {
  if (!ms_active(flags, o)) return;
  long long n1 = 0, s0 = 0, s1 = 0, n0 = 0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += (int64_t)gridDim.x * blockDim.x) {
    const int v = g[b];
    if (s[b]) {
      ++n1;
      s1 += v;
    } else {
      ++n0;
      s0 += v;
    }
  }
  for (int k = 16; k > 0; k >>= 1) {
    n0 += __shfl_xor_sync(0xffffffffu, n0, k);
    s0 += __shfl_xor_sync(0xffffffffu, s0, k);
    n1 += __shfl_xor_sync(0xffffffffu, n1, k);
    s1 += __shfl_xor_sync(0xffffffffu, s1, k);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sums + 4 * o + 0, (unsigned long long)n0);
    atomicAdd(sums + 4 * o + 1, (unsigned long long)s0);
    atomicAdd(sums + 4 * o + 2, (unsigned long long)n1);
    atomicAdd(sums + 4 * o + 3, (unsigned long long)s1);
  }
}

// Phase values, data weights, and the start of the inner iteration (u = s, p = 0).
template <typename R>
__global__ void k_ms_start(const int32_t* __restrict__ g, const uint8_t* __restrict__ s, int64_t nbox,
                           const unsigned long long* sums, int32_t* flags, double* c, int o, R* __restrict__ w,
                           R* __restrict__ u, R* __restrict__ ub, R* __restrict__ p) {
  if (!ms_active(flags, o)) return;
  const unsigned long long n0 = sums[4 * o], n1 = sums[4 * o + 2];
  if (n0 == 0 || n1 == 0) {  // one phase is empty: s stays as it is
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[0] = 1;
    return;
  }
  const double c0 = (double)(long long)sums[4 * o + 1] / (double)n0;
  const double c1 = (double)(long long)sums[4 * o + 3] / (double)n1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c[0] = c0;
    c[1] = c1;
  }
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += (int64_t)gridDim.x * blockDim.x) {
    const double gv = (double)g[b];
    const double d1 = __dsub_rn(gv, c1), d0 = __dsub_rn(gv, c0);
    w[b] = (R)__dsub_rn(__dmul_rn(d1, d1), __dmul_rn(d0, d0));
    const R v = s[b] ? (R)1 : (R)0;
    u[b] = v;
    ub[b] = v;
    p[3 * b] = p[3 * b + 1] = p[3 * b + 2] = (R)0;
  }
}

// Dual step: p_f <- clip(p_f + sigma (ubar_{b+e} - ubar_b), -nu, nu) for the
// three faces (b, b + e) of every box b.
template <typename R>
__global__ void k_ms_dual(const R* __restrict__ ub, R* __restrict__ p, int nx, int ny, int nz, R sigma, R nu,
                          const int32_t* flags, int o) {
  if (!ms_active(flags, o)) return;
  const int64_t nxy = (int64_t)nx * ny, nbox = nxy * nz;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / nxy);
    const int64_t nb[3] = {b - x + (x == nx - 1 ? 0 : x + 1), b + (int64_t)((y == ny - 1 ? 0 : y + 1) - y) * nx,
                           b + (int64_t)((z == nz - 1 ? 0 : z + 1) - z) * nxy};
    const R ubb = ub[b];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const R q = r_add(p[3 * b + e], r_mul(sigma, r_sub(ub[nb[e]], ubb)));
      p[3 * b + e] = q < -nu ? -nu : (q > nu ? nu : q);
    }
  }
}

// Primal step: u' = clip(u - tau ((D^T p)_b + w_b), 0, 1), ubar = 2 u' - u.
template <typename R>
__global__ void k_ms_primal(const R* __restrict__ p, const R* __restrict__ w, R* __restrict__ u, R* __restrict__ ub,
                            int nx, int ny, int nz, R tau, const int32_t* flags, int o) {
  if (!ms_active(flags, o)) return;
  const int64_t nxy = (int64_t)nx * ny, nbox = nxy * nz;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / nxy);
    const int64_t pb[3] = {b - x + (x == 0 ? nx - 1 : x - 1), b + (int64_t)((y == 0 ? ny - 1 : y - 1) - y) * nx,
                           b + (int64_t)((z == 0 ? nz - 1 : z - 1) - z) * nxy};
    R dtp = (R)0;
#pragma unroll
    for (int e = 0; e < 3; ++e) dtp = r_add(dtp, r_sub(p[3 * pb[e] + e], p[3 * b + e]));
    const R ub0 = u[b];
    R v = r_sub(ub0, r_mul(tau, r_add(dtp, w[b])));
    v = v < (R)0 ? (R)0 : (v > (R)1 ? (R)1 : v);
    ub[b] = r_sub(r_mul((R)2, v), ub0);
    u[b] = v;
  }
}

// s = (u >= 1/2); flags[o + 1] = 1 if any box changed.
template <typename R>
__global__ void k_ms_threshold(const R* __restrict__ u, uint8_t* __restrict__ s, int64_t nbox, int32_t* flags,
                               int o) {
  if (!ms_active(flags, o)) return;
  bool changed = false;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t t = u[b] >= (R)0.5 ? 1 : 0;
    changed |= t != s[b];
    s[b] = t;
  }
  if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) flags[o + 1] = 1;
}

template <typename R>
int ms_run(dcm_ctx* ctx, const int32_t* count, uint8_t* s, cudaStream_t st) {
  const int nx = (int)ctx->nh[0], ny = (int)ctx->nh[1], nz = (int)ctx->nh[2];
  const int64_t nbox = ctx->nbox;
  const int outer = ctx->p.ms_outer, inner = ctx->p.ms_inner;
  const unsigned grid = (unsigned)std::min<int64_t>((nbox + 255) / 256, 152 * 8);
  R* u = (R*)ctx->ms_u;
  R* ub = (R*)ctx->ms_ub;
  R* p = (R*)ctx->ms_p;
  R* w = (R*)ctx->ms_w;
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->ms_flags, 0, sizeof(int32_t) * (size_t)(outer + 2), st));
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->ms_sums, 0, sizeof(unsigned long long) * 4 * (size_t)outer, st));
  for (int o = 0; o < outer; ++o) {
    DCM_LAUNCH(ctx, k_ms_sums, grid, 256, 0, st, count, s, nbox, ctx->ms_sums, ctx->ms_flags, o);
    DCM_LAUNCH(ctx, k_ms_start<R>, grid, 256, 0, st, count, s, nbox, ctx->ms_sums, ctx->ms_flags, ctx->ms_c, o, w, u,
               ub, p);
    for (int it = 0; it < inner; ++it) {
      DCM_LAUNCH(ctx, k_ms_dual<R>, grid, 256, 0, st, ub, p, nx, ny, nz, (R)kMsSigma, (R)ctx->p.ms_nu,
                 ctx->ms_flags, o);
      DCM_LAUNCH(ctx, k_ms_primal<R>, grid, 256, 0, st, p, w, u, ub, nx, ny, nz, (R)kMsTau, ctx->ms_flags, o);
    }
    DCM_LAUNCH(ctx, k_ms_threshold<R>, grid, 256, 0, st, u, s, nbox, ctx->ms_flags, o);
  }
  return check_launch(ctx, "ms_segment");
}

}  // namespace

int ms_segment(dcm_ctx* ctx, const int32_t* count, uint8_t* s, cudaStream_t st) {
  if (ctx->precision == DCM_PREC_FP64) return ms_run<double>(ctx, count, s, st);
  return ms_run<float>(ctx, count, s, st);
}

}  // namespace dcm
