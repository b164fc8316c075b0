// Deterministic final reduction of per-block FP64 partials: one block per
// quantity, fixed strided assignment and a fixed tree, so totals do not
// depend on scheduling.
#include "dcm_internal.cuh"

namespace dcm {

__global__ void __launch_bounds__(256) k_reduce_partials(const double* __restrict__ part, int64_t nblk,
                                                         double* __restrict__ out, int accumulate) {
  const double* p = part + (int64_t)blockIdx.x * nblk;
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < nblk; k += blockDim.x) s += p[k];
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = accumulate ? out[blockIdx.x] + sh[0] : sh[0];
}

int reduce_partials(dcm_ctx* ctx, const double* part, int64_t nblk, int nq, double* out, bool accumulate,
                    cudaStream_t st) {
  DCM_LAUNCH(ctx, k_reduce_partials, nq, 256, 0, st, part, nblk, out, accumulate ? 1 : 0);
  return check_launch(ctx, "reduce_partials");
}

}  // namespace dcm
