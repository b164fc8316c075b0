// Launch order of tiles by decreasing cost.
//
// The per-particle kernels (forces, adjoint) run one block per tile of
// consecutive cell-sorted particles.  A tile costs about as much as its
// widest walk (the largest cutoff, or reach, among its particles), and the
// costly tiles form bands near the interfaces, one of them close to the end
// of the cell order.  Blocks start roughly in launch order, so a launch in
// which the first blocks take the costly tiles ends on cheap ones instead of
// waiting for a costly straggler.
//
// The order is a stable counting sort of the tiles over kTileBins bins of
// their key (the widest tile first; within a bin by tile index, so that
// neighbouring tiles still run side by side): a key kernel writes each
// tile's bin and counts it per chunk of kTileChunk tiles, tile_order_finish
// scans the counts bin-major and places every tile.  A tile keeps its
// particles and its output slots wherever it runs, so results do not depend
// on the order.
#pragma once

#include "dcm_internal.cuh"

namespace dcm {

struct TileOrder {
  int32_t* order;  // [ntile]: the tile each block takes
  int32_t* key;    // [ntile]: the bin of each tile (0 = widest)
  int32_t* cnt;    // [kTileBins][nchunk]: tiles of each bin per chunk, scanned in place
  int64_t ntile, nchunk;
};

inline TileOrder tile_order_layout(int32_t* scratch, int64_t ntile) {
  TileOrder t;
  t.ntile = ntile;
  t.nchunk = tile_chunks(ntile);
  t.order = scratch;
  t.key = scratch + ntile;
  t.cnt = scratch + 2 * ntile;
  return t;
}

// Whether ordering pays for a launch of ntile blocks of `kernel` with
// `threads` threads: at most kTileOrderWaves waves of resident blocks, where
// the last wave is a large share of the launch.  Over many waves the tail is
// small and launching neighbouring tiles apart costs more than it saves
// (measured with the packed force kernel: 260K particles, 1.7 waves, 0.357
// -> 0.31 ms; 16M, 100 waves, 5.63 -> 5.80 ms; the 64-replica batch, 14.6
// waves of 256-thread blocks, 1.35 -> 1.29 ms).
constexpr int kTileOrderWaves = 16;
bool tile_order_pays(const void* kernel, int threads, int64_t ntile);

// Zero the counts (before the key kernel).
int tile_order_begin(dcm_ctx* ctx, const TileOrder& t, cudaStream_t st);
// Scan the counts and write the order (after the key kernel).
int tile_order_finish(dcm_ctx* ctx, const TileOrder& t, cudaStream_t st);

// Called by every thread of a key kernel that runs one block per tile (tile =
// blockIdx.x, at most 1024 threads): v is the thread's particle's walk radius
// (0 past the end), top the largest possible one.
__device__ __forceinline__ void tile_key_of_block(float v, float top, int32_t* __restrict__ key,
                                                  int32_t* __restrict__ cnt, int64_t nchunk) {
  __shared__ float wmax[32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = wmax[0];
    for (int w = 1; w < (int)((blockDim.x + 31) >> 5); ++w) m = fmaxf(m, wmax[w]);
    int b = m > 0.f ? (int)(m / top * (float)kTileBins) : 0;  // NaN and negatives: bin 0
    b = b < 0 ? 0 : (b > kTileBins - 1 ? kTileBins - 1 : b);
    const int k = kTileBins - 1 - b;
    key[blockIdx.x] = k;
    atomicAdd(cnt + (int64_t)k * nchunk + blockIdx.x / kTileChunk, 1);
  }
}

}  // namespace dcm
