// Deterministic reduction of per-block FP64 partials: a fixed number of
// first-level blocks each sums a fixed contiguous chunk in a fixed order, then
// one block sums the chunk totals, so totals do not depend on scheduling.
#include "dcm_internal.cuh"

namespace dcm {

constexpr int kRedChunks = 256;  // first-level blocks per quantity

__device__ __forceinline__ double block_sum_d(double s) {
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  return sh[0];
}

// grid (kRedChunks, nq): chunk c of quantity q -> tmp[q * kRedChunks + c]
__global__ void __launch_bounds__(256) k_reduce_level1(const double* __restrict__ part, int64_t nblk,
                                                       double* __restrict__ tmp) {
  const double* p = part + (int64_t)blockIdx.y * nblk;
  int64_t per = (nblk + kRedChunks - 1) / kRedChunks;
  int64_t b0 = (int64_t)blockIdx.x * per, b1 = b0 + per < nblk ? b0 + per : nblk;
  double s = 0.0;
  for (int64_t k = b0 + threadIdx.x; k < b1; k += blockDim.x) s += p[k];
  double t = block_sum_d(s);
  if (threadIdx.x == 0) tmp[blockIdx.y * kRedChunks + blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_reduce_level2(const double* __restrict__ tmp, double* __restrict__ out,
                                                       int accumulate) {
  double s = tmp[blockIdx.x * kRedChunks + threadIdx.x];  // blockDim == kRedChunks
  double t = block_sum_d(s);
  if (threadIdx.x == 0) out[blockIdx.x] = accumulate ? out[blockIdx.x] + t : t;
}

int reduce_partials(dcm_ctx* ctx, const double* part, int64_t nblk, int nq, double* out, bool accumulate,
                    cudaStream_t st) {
  if (nq > 8) return set_error(ctx, DCM_ERR_INVALID_ARG, "reduce_partials: too many quantities");
  DCM_LAUNCH(ctx, k_reduce_level1, dim3(kRedChunks, nq), 256, 0, st, part, nblk, ctx->red_tmp);
  DCM_LAUNCH(ctx, k_reduce_level2, nq, kRedChunks, 0, st, ctx->red_tmp, out, accumulate ? 1 : 0);
  return check_launch(ctx, "reduce_partials");
}

}  // namespace dcm
