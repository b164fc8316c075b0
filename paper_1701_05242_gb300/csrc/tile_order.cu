// Stable counting sort of tiles by their cost bin (see tile_order.cuh).
#include "tile_order.cuh"

#include <mutex>
#include <vector>

namespace dcm {

namespace {

// Exclusive scan, in place, of the M = kTileBins * nchunk bin counts in
// bin-major order (bin 0 of every chunk first): one block, each thread a
// contiguous run of the counts.
__global__ void __launch_bounds__(1024) k_tile_scan(int32_t* __restrict__ cnt, int64_t m) {
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t per = (m + 1023) / 1024;
  const int64_t lo = (int64_t)tid * per, hi = lo + per < m ? lo + per : m;
  int s = 0;
  for (int64_t i = lo; i < hi; ++i) s += cnt[i];
  int x = s;  // inclusive scan over the warp
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wsum[lane] = t;  // inclusive warp totals
  }
  __syncthreads();
  int run = x - s + (w > 0 ? wsum[w - 1] : 0);
  for (int64_t i = lo; i < hi; ++i) {
    const int c = cnt[i];
    cnt[i] = run;
    run += c;
  }
}

// One block per chunk of kTileChunk tiles: a tile's slot is its bin's start
// for the chunk plus the tiles of the same bin before it in the chunk (ranks
// from the warps' matching keys, then the earlier warps' counts).
__global__ void __launch_bounds__(kTileChunk) k_tile_place(int64_t ntile, const int32_t* __restrict__ key,
                                                          const int32_t* __restrict__ base, int64_t nchunk,
                                                          int32_t* __restrict__ order) {
  __shared__ int wc[kTileChunk / 32][kTileBins];
  for (int q = threadIdx.x; q < (kTileChunk / 32) * kTileBins; q += blockDim.x) wc[q / kTileBins][q % kTileBins] = 0;
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * kTileChunk + threadIdx.x;
  const int k = t < ntile ? key[t] : -1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned same = __match_any_sync(0xffffffffu, k);
  const int rank = __popc(same & ((1u << lane) - 1u));
  if (k >= 0 && rank == 0) wc[w][k] = __popc(same);
  __syncthreads();
  if (k >= 0) {
    int off = rank;
    for (int v = 0; v < w; ++v) off += wc[v][k];
    order[base[(int64_t)k * nchunk + blockIdx.x] + off] = (int32_t)t;
  }
}

}  // namespace

// Resident blocks of (kernel, threads) on the current device, remembered per
// device (the query is made once per kernel, not once per launch).
static int64_t resident_blocks(const void* kernel, int threads) {
  struct Entry {
    const void* kernel;
    int threads, dev;
    int64_t blocks;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(mu);
  for (const Entry& e : cache)
    if (e.kernel == kernel && e.threads == threads && e.dev == dev) return e.blocks;
  int sms = 0, nb = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess) {
    cudaGetLastError();  // a failed query only turns the order off; it is not a launch error
    return 0;
  }
  cache.push_back(Entry{kernel, threads, dev, (int64_t)nb * sms});
  return (int64_t)nb * sms;
}

bool tile_order_pays(const void* kernel, int threads, int64_t ntile) {
  const int64_t r = resident_blocks(kernel, threads);
  return r > 0 && ntile <= (int64_t)kTileOrderWaves * r;
}

int tile_order_begin(dcm_ctx* ctx, const TileOrder& t, cudaStream_t st) {
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(t.cnt, 0, sizeof(int32_t) * kTileBins * t.nchunk, st));
  return DCM_OK;
}

int tile_order_finish(dcm_ctx* ctx, const TileOrder& t, cudaStream_t st) {
  DCM_LAUNCH(ctx, k_tile_scan, 1, 1024, 0, st, t.cnt, (int64_t)kTileBins * t.nchunk);
  DCM_LAUNCH(ctx, k_tile_place, (unsigned)t.nchunk, kTileChunk, 0, st, t.ntile, (const int32_t*)t.key,
             (const int32_t*)t.cnt, t.nchunk, t.order);
  return DCM_OK;
}

}  // namespace dcm
