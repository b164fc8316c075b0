// Interface detection (Section 2.1, Eq. 4): gray-scale volume from box counts,
// two-phase segmentation by an integer 2-means threshold (refined, with
// params.segmentation = 1, by the regularised segmentation of segment_ms.cu),
// interface boxes.
//
// All integer arithmetic, so the result is bit-identical to any correct
// evaluation: the (2w+1)^3 box sum is computed as three separable 1-D periodic
// sums, and the 2-means iteration runs on a histogram of the box sums (same
// counts and sums as scanning the volume, in one pass instead of one per
// iteration).
#include <algorithm>
#include <climits>

#include "dcm_internal.cuh"

namespace dcm {

// out[x,y,z] = sum_{a=-w..w} in[x+a (periodic along axis), y, z]
template <int AXIS>
__global__ void k_box_sum_axis(const int32_t* __restrict__ in, int32_t* __restrict__ out, int nx, int ny, int nz,
                               int w) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t nbox = (int64_t)nx * ny * nz;
  if (b >= nbox) return;
  int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / ((int64_t)nx * ny));
  int n = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
  int c = AXIS == 0 ? x : (AXIS == 1 ? y : z);
  int64_t stride = AXIS == 0 ? 1 : (AXIS == 1 ? nx : (int64_t)nx * ny);
  int64_t base = b - (int64_t)c * stride;
  int s = 0;
  for (int a = -w; a <= w; ++a) {
    int k = c + a;
    k %= n;
    if (k < 0) k += n;
    s += in[base + (int64_t)k * stride];
  }
  out[b] = s;
}

__global__ void k_minmax_init(int32_t* thr) {
  thr[0] = INT_MAX;
  thr[1] = INT_MIN;
}

__global__ void k_minmax(const int32_t* __restrict__ g, int64_t nbox, int32_t* thr) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int lo = INT_MAX, hi = INT_MIN;
  for (; b < nbox; b += (int64_t)gridDim.x * blockDim.x) {
    int v = g[b];
    lo = min(lo, v);
    hi = max(hi, v);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(thr, lo);
    atomicMax(thr + 1, hi);
  }
}

// Histogram of the box sums over [gmin, gmax]: per-block shared-memory
// histogram when the range fits (kSmemBins), else global atomics.
constexpr int kSmemBins = 8192;

__global__ void k_value_hist(const int32_t* __restrict__ g, int64_t nbox, const int32_t* thr, int32_t* hist,
                             int32_t* status) {
  __shared__ int32_t sh[kSmemBins];
  int gmin = thr[0], gmax = thr[1];
  if ((int64_t)gmax - gmin >= kHistCap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(status, DCM_ERR_CAPACITY);
    return;
  }
  int range = gmax - gmin + 1;
  if (range <= kSmemBins) {
    for (int k = threadIdx.x; k < range; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += (int64_t)gridDim.x * blockDim.x)
      atomicAdd(sh + (g[b] - gmin), 1);
    __syncthreads();
    for (int k = threadIdx.x; k < range; k += blockDim.x)
      if (sh[k]) atomicAdd(hist + k, sh[k]);
  } else {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += (int64_t)gridDim.x * blockDim.x)
      atomicAdd(hist + (g[b] - gmin), 1);
  }
}

__device__ long long block_sum_ll(long long v, long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  long long t = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  return t;
}

// One block: integer 2-means (Lloyd) on the histogram of box sums.
//   T0 = floor((gmin + gmax) / 2); repeat: class 0 = values < T, class 1 = >= T;
//   T <- floor((S0 n1 + S1 n0) / (2 n0 n1)) + 1 until T repeats (<= max_iter).
// One empty class: T = gmax + 1 (no interface).  fixed >= 0 bypasses it.
__global__ void k_two_means(const int32_t* __restrict__ hist, int32_t* thr, int max_iter, int fixed,
                            int32_t* t_out) {
  __shared__ long long sh[32];
  __shared__ int T_sh;
  int gmin = thr[0], gmax = thr[1];
  if (fixed >= 0) {
    if (threadIdx.x == 0) {
      thr[2] = fixed;
      if (t_out) *t_out = fixed;
    }
    return;
  }
  if ((int64_t)gmax - gmin >= kHistCap) return;  // capacity error already raised
  int R = gmax - gmin + 1;
  if (threadIdx.x == 0) T_sh = (int)(((long long)gmin + gmax) / 2);
  __syncthreads();
  for (int it = 0; it < max_iter; ++it) {
    int T = T_sh;
    long long n0 = 0, n1 = 0, s0 = 0, s1 = 0;
    for (int k = threadIdx.x; k < R; k += blockDim.x) {
      long long c = hist[k], v = (long long)(gmin + k);
      if (gmin + k < T) {
        n0 += c;
        s0 += c * v;
      } else {
        n1 += c;
        s1 += c * v;
      }
    }
    n0 = block_sum_ll(n0, sh);
    n1 = block_sum_ll(n1, sh);
    s0 = block_sum_ll(s0, sh);
    s1 = block_sum_ll(s1, sh);
    __syncthreads();
    int stop = 0;
    if (n0 == 0 || n1 == 0) {
      if (threadIdx.x == 0) T_sh = gmax + 1;
      stop = 1;
    } else {
      int Tn = (int)((s0 * n1 + s1 * n0) / (2 * n0 * n1) + 1);
      if (Tn == T) stop = 1;
      if (threadIdx.x == 0) T_sh = Tn;
    }
    __syncthreads();
    if (stop) break;
  }
  if (threadIdx.x == 0) {
    thr[2] = T_sh;
    if (t_out) *t_out = T_sh;
  }
}

// s = (g >= T); interface = s and some face neighbour below T (periodic).
__global__ void k_segment(const int32_t* __restrict__ g, int nx, int ny, int nz, const int32_t* thr,
                          uint8_t* __restrict__ s, uint8_t* __restrict__ iface) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t nxy = (int64_t)nx * ny;
  if (b >= nxy * nz) return;
  int T = thr[2];
  int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / nxy);
  int me = g[b] >= T;
  int f = 0;
  if (me) {
    int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    int64_t row = (int64_t)nx * (y + (int64_t)ny * z);
    f |= g[row + xm] < T;
    f |= g[row + xp] < T;
    f |= g[x + nx * (ym + (int64_t)ny * z)] < T;
    f |= g[x + nx * (yp + (int64_t)ny * z)] < T;
    f |= g[x + nx * (y + (int64_t)ny * zm)] < T;
    f |= g[x + nx * (y + (int64_t)ny * zp)] < T;
  }
  s[b] = (uint8_t)me;
  iface[b] = (uint8_t)f;
}

int detect_interface(dcm_ctx* ctx, const int32_t* box_count, uint8_t* s, uint8_t* iface, int32_t* threshold,
                     int32_t* g_out, cudaStream_t st) {
  int nx = (int)ctx->nh[0], ny = (int)ctx->nh[1], nz = (int)ctx->nh[2];
  int64_t nbox = ctx->nbox;
  int w = ctx->p.smooth_w;
  int32_t* g = g_out ? g_out : ctx->g;
  unsigned nb = (unsigned)((nbox + 255) / 256);
  // separable box sum: x into g, y into g_tmp, z back into g
  DCM_LAUNCH(ctx, k_box_sum_axis<0>, nb, 256, 0, st, box_count, g, nx, ny, nz, w);
  DCM_LAUNCH(ctx, k_box_sum_axis<1>, nb, 256, 0, st, g, ctx->g_tmp, nx, ny, nz, w);
  DCM_LAUNCH(ctx, k_box_sum_axis<2>, nb, 256, 0, st, ctx->g_tmp, g, nx, ny, nz, w);
  if (ctx->p.threshold < 0) {
    DCM_LAUNCH(ctx, k_minmax_init, 1, 1, 0, st, ctx->thr);
    int nred = (int)std::min<int64_t>((nbox + 255) / 256, 152 * 4);
    DCM_LAUNCH(ctx, k_minmax, nred, 256, 0, st, g, nbox, ctx->thr);
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->hist, 0, sizeof(int32_t) * kHistCap, st));
    DCM_LAUNCH(ctx, k_value_hist, nred, 256, 0, st, g, nbox, ctx->thr, ctx->hist, ctx->status);
  }
  DCM_LAUNCH(ctx, k_two_means, 1, 1024, 0, st, ctx->hist, ctx->thr, 64, ctx->p.threshold, threshold);
  if (ctx->p.min_component > 0) {
    // segment (and refine) into scratch, then the filtered S and its interface into s, iface
    DCM_LAUNCH(ctx, k_segment, nb, 256, 0, st, g, nx, ny, nz, ctx->thr, ctx->cc_s0, iface);
    int r = check_launch(ctx, "detect_interface");
    if (r) return r;
    if (ctx->p.segmentation && (r = ms_segment(ctx, box_count, ctx->cc_s0, st))) return r;
    return remove_small_components(ctx, ctx->cc_s0, s, iface, st);
  }
  DCM_LAUNCH(ctx, k_segment, nb, 256, 0, st, g, nx, ny, nz, ctx->thr, s, iface);
  if (ctx->p.segmentation) {
    // the regularised segmentation of the counts refines the threshold's S
    int r = ms_segment(ctx, box_count, s, st);
    if (r) return r;
    interface_of(ctx, s, iface, st);
  }
  return check_launch(ctx, "detect_interface");
}

}  // namespace dcm
