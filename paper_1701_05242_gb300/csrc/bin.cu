// Binning into cells (Sections 2.1 and 2.3): exact cell index, counts,
// exclusive scan of the counts, and a stable scatter.
//
// Stability without a global sort: atomics give every particle a provisional
// rank inside its cell, the scatter places it there, and one thread per cell
// then insertion-sorts the cell's (few) entries by input index.  The result
// is the unique stable order, independent of atomic timing.
#include "dcm_internal.cuh"

namespace dcm {

template <typename R>
__global__ void k_count(int64_t n, const typename RT<R>::R4* __restrict__ pos, Grid<R> g,
                        int32_t* __restrict__ cell, int32_t* __restrict__ slot, int32_t* __restrict__ count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto p = ldg4(pos + i);
  int cx = cell_coord<R>(p.x, g.edge_x, g.inv_edge_x, g.n[0]);
  int cy = cell_coord<R>(p.y, g.edge, g.inv_edge, g.n[1]);
  int cz = cell_coord<R>(p.z, g.edge, g.inv_edge, g.n[2]);
  int c = cx + g.n[0] * (cy + g.n[1] * cz);
  int r = atomicAdd(count + c, 1);
  if (cell) cell[i] = c;
  if (slot) slot[i] = r;
}

// Block-wide exclusive scan helpers (1024 threads, 32 warps).
__device__ __forceinline__ int warp_incl_scan(int v) {
  int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Returns the exclusive prefix of v over the block; *total receives the sum.
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int warp_sums[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) warp_sums[w] = inc;
  __syncthreads();
  if (w == 0) {
    int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
    s = warp_incl_scan(s);
    warp_sums[lane] = s;
  }
  __syncthreads();
  int base = w > 0 ? warp_sums[w - 1] : 0;
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + inc - v;
}

// Single-pass exclusive scan with decoupled look-back (Merrill and
// Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back",
// 2016).  Each block takes the next tile of kScanTile items by a ticket (so
// every tile it waits for belongs to a block that is already running),
// scans it, publishes the tile's sum, and then its first warp walks back
// over the preceding tiles' words, 32 at a time, adding their sums until it
// meets a tile that has published its inclusive prefix.  A word packs its
// kind (bits 62-63: 0 not yet published, 1 the tile's sum, 2 the inclusive
// prefix) and its value (bits 0-31) so that one 64-bit store publishes both.
// Every wait is bounded by a poll count; a block that runs out records
// DCM_ERR_TIMEOUT in the device status and carries on with prefix 0 (the
// caller reads the status).  state[0 .. ntiles] must be zero at launch
// (state[ntiles] is the ticket counter).
constexpr unsigned long long kScanSum = 1ull << 62, kScanPrefix = 2ull << 62;
constexpr int64_t kScanMaxPolls = 1 << 20;  // about a second of polls

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__global__ void __launch_bounds__(kScanBlock) k_scan_lookback(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                              int64_t n, unsigned long long* state, int64_t ntiles,
                                                              int32_t* status) {
  __shared__ int64_t tile_sh;
  __shared__ int prefix_sh;
  if (threadIdx.x == 0) tile_sh = (int64_t)atomicAdd(state + ntiles, 1ull);
  __syncthreads();
  const int64_t t = tile_sh;
  const int64_t base = t * kScanTile + (int64_t)threadIdx.x * kScanItems;
  static_assert(kScanItems % 4 == 0, "whole 16-byte groups per thread");
  constexpr int kQ = kScanItems / 4;
  const bool vec = ((((uintptr_t)in) | ((uintptr_t)out)) & 15) == 0;
  int4 v[kQ];
  int sum = 0;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int64_t b = base + 4 * q;
    v[q] = make_int4(0, 0, 0, 0);
    if (vec && b + 4 <= n) {
      v[q] = *reinterpret_cast<const int4*>(in + b);
    } else if (b < n) {
      v[q].x = in[b];
      v[q].y = b + 1 < n ? in[b + 1] : 0;
      v[q].z = b + 2 < n ? in[b + 2] : 0;
      v[q].w = b + 3 < n ? in[b + 3] : 0;
    }
    sum += v[q].x + v[q].y + v[q].z + v[q].w;
  }
  int total;
  const int run = block_excl_scan(sum, &total);
  if (threadIdx.x < 32) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x;
    int prefix = 0;
    if (t == 0) {
      if (lane == 0) atomicExch(state, kScanPrefix | (unsigned)total);
    } else {
      if (lane == 0) atomicExch(state + t, kScanSum | (unsigned)total);
      int64_t look = t - 1;
      int64_t polls = 0;
      for (;;) {
        const int64_t k = look - lane;
        const unsigned long long wv = k >= 0 ? ld_word(state + k) : kScanPrefix;
        if (__any_sync(full, (wv >> 62) == 0)) {
          if (++polls > kScanMaxPolls) {
            if (lane == 0) raise_status(status, DCM_ERR_TIMEOUT);
            prefix = 0;
            break;
          }
          __nanosleep(32);
          continue;
        }
        // the nearest inclusive prefix in the window ends the walk
        const unsigned pre = __ballot_sync(full, (wv >> 62) == 2);
        const int stop = pre ? __ffs(pre) - 1 : 31;
        prefix += __reduce_add_sync(full, lane <= stop ? (unsigned)(wv & 0xffffffffull) : 0u);
        if (pre) break;
        look -= 32;
      }
      if (lane == 0) atomicExch(state + t, kScanPrefix | (unsigned)(prefix + total));
    }
    if (lane == 0) prefix_sh = prefix;
  }
  __syncthreads();
  int ex = prefix_sh + run;
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int64_t b = base + 4 * q;
    const int4 o = make_int4(ex, ex + v[q].x, ex + v[q].x + v[q].y, ex + v[q].x + v[q].y + v[q].z);
    if (vec && b + 4 <= n) {
      *reinterpret_cast<int4*>(out + b) = o;
    } else if (b < n) {
      out[b] = o.x;
      if (b + 1 < n) out[b + 1] = o.y;
      if (b + 2 < n) out[b + 2] = o.z;
      if (b + 3 < n) out[b + 3] = o.w;
    }
    ex = o.w + v[q].w;
  }
  if (t == ntiles - 1 && threadIdx.x == 0) out[n] = prefix_sh + total;
}

int exclusive_scan(dcm_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles > ctx->scan_cap) return set_error(ctx, DCM_ERR_CAPACITY, "scan of %lld items exceeds scratch", (long long)n);
  if (tiles == 0) {
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, sizeof(int32_t), st));
    return DCM_OK;
  }
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->scan_state, 0, sizeof(unsigned long long) * (size_t)(tiles + 1), st));
  DCM_LAUNCH(ctx, k_scan_lookback, (unsigned)tiles, kScanBlock, 0, st, in, out, n, ctx->scan_state, tiles, ctx->status);
  return check_launch(ctx, "exclusive_scan");
}

// The scan's failure path: two tiles of zeros with the first tile's block
// left out (the ticket counter starts at 1), so the one block launched takes
// tile 1 and its look-back waits for a word that is never published.
int scan_wait_selftest(dcm_ctx* ctx, cudaStream_t st) {
  int32_t* buf = nullptr;
  unsigned long long* state = nullptr;
  const int64_t n = 2 * (int64_t)kScanTile;
  if (cudaMalloc((void**)&buf, sizeof(int32_t) * (size_t)(2 * n + 1)) != cudaSuccess)
    return set_error(ctx, DCM_ERR_NOMEM, "scan self-test buffer");
  if (cudaMalloc((void**)&state, sizeof(unsigned long long) * 3) != cudaSuccess) {
    cudaFree(buf);
    return set_error(ctx, DCM_ERR_NOMEM, "scan self-test state");
  }
  int r = DCM_OK;
  if (cudaMemsetAsync(buf, 0, sizeof(int32_t) * (size_t)(2 * n + 1), st) != cudaSuccess ||
      cudaMemsetAsync(state, 0, sizeof(unsigned long long) * 3, st) != cudaSuccess ||
      cudaMemsetAsync(state + 2, 1, 1, st) != cudaSuccess)  // ticket counter = 1 (little-endian low byte)
    r = set_error(ctx, DCM_ERR_CUDA, "scan self-test set-up");
  if (r == DCM_OK) {
    k_scan_lookback<<<1, kScanBlock, 0, st>>>(buf, buf + n, n, state, 2, ctx->status);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      r = set_error(ctx, DCM_ERR_CUDA, "scan self-test launch");
  }
  cudaFree(buf);
  cudaFree(state);
  return r;
}

__global__ void k_scatter(int64_t n, const int32_t* __restrict__ cell, const int32_t* __restrict__ slot,
                          const int32_t* __restrict__ start, int32_t* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  perm[start[cell[i]] + slot[i]] = (int32_t)i;
}

// Four particles per thread (cell and slot 16-byte aligned): one 16-byte load
// of each and four independent cell-start loads in flight.
__global__ void k_scatter4(int64_t n, const int32_t* __restrict__ cell, const int32_t* __restrict__ slot,
                           const int32_t* __restrict__ start, int32_t* __restrict__ perm) {
  const int64_t i = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  if (i + 4 <= n) {
    const int4 c = *reinterpret_cast<const int4*>(cell + i), q = *reinterpret_cast<const int4*>(slot + i);
    const int s0 = start[c.x], s1 = start[c.y], s2 = start[c.z], s3 = start[c.w];
    perm[s0 + q.x] = (int32_t)i;
    perm[s1 + q.y] = (int32_t)(i + 1);
    perm[s2 + q.z] = (int32_t)(i + 2);
    perm[s3 + q.w] = (int32_t)(i + 3);
  } else {
    for (int64_t k = i; k < n; ++k) perm[start[cell[k]] + slot[k]] = (int32_t)k;
  }
}

static void launch_scatter(dcm_ctx* ctx, int64_t n, const int32_t* cell, const int32_t* slot, const int32_t* start,
                           int32_t* perm, cudaStream_t st) {
  if ((((uintptr_t)cell | (uintptr_t)slot) & 15) == 0)
    DCM_LAUNCH(ctx, k_scatter4, (unsigned)(((n + 3) / 4 + 255) / 256), 256, 0, st, n, cell, slot, start, perm);
  else
    DCM_LAUNCH(ctx, k_scatter, (unsigned)((n + 255) / 256), 256, 0, st, n, cell, slot, start, perm);
}

// Insertion sort of one cell's entries perm[b .. e) by input index.
__device__ __forceinline__ void sort_cell(int b, int e, int32_t* __restrict__ perm) {
  for (int k = b + 1; k < e; ++k) {
    int v = perm[k];
    int j = k - 1;
    while (j >= b && perm[j] > v) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = v;
  }
}

// One thread per cell.
__global__ void k_cell_sort(int64_t ncell, const int32_t* __restrict__ start, int32_t* __restrict__ perm) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  sort_cell(start[c], start[c + 1], perm);
}

// Eight cells per thread, their nine starts from two 16-byte loads and one
// more (start 16-byte aligned; most cells hold at most one particle, so the
// pass is mostly a read of the starts; eight per thread keep more of those
// reads in flight than four: 66 against 82 us at 49M cells).
__global__ void k_cell_sort8(int64_t ncell, const int32_t* __restrict__ start, int32_t* __restrict__ perm) {
  const int64_t c = 8 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (c >= ncell) return;
  int s[9];
  if (c + 8 <= ncell) {
    const int4 v = *reinterpret_cast<const int4*>(start + c), u = *reinterpret_cast<const int4*>(start + c + 4);
    s[0] = v.x;
    s[1] = v.y;
    s[2] = v.z;
    s[3] = v.w;
    s[4] = u.x;
    s[5] = u.y;
    s[6] = u.z;
    s[7] = u.w;
    s[8] = start[c + 8];
  } else {
    for (int q = 0; q < 9; ++q) s[q] = start[min(c + q, ncell)];
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) sort_cell(s[q], s[q + 1], perm);
}

static void launch_cell_sort(dcm_ctx* ctx, int64_t ncell, const int32_t* start, int32_t* perm, cudaStream_t st) {
  if (((uintptr_t)start & 15) == 0)
    DCM_LAUNCH(ctx, k_cell_sort8, (unsigned)(((ncell + 7) / 8 + 255) / 256), 256, 0, st, ncell, start, perm);
  else
    DCM_LAUNCH(ctx, k_cell_sort, (unsigned)((ncell + 255) / 256), 256, 0, st, ncell, start, perm);
}

template <typename V>
__global__ void k_gather(int64_t n, const int32_t* __restrict__ perm, const V* __restrict__ src, V* __restrict__ dst) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  dst[k] = src[perm[k]];
}

template <typename R>
int bin_particles(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const Grid<R>& grid, int32_t* cell,
                  int32_t* cell_start, int32_t* perm, typename RT<R>::R4* pos_sorted, cudaStream_t st) {
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cell_count, 0, sizeof(int32_t) * grid.ncell, st));
  if (n > 0) {
    unsigned nb = (unsigned)((n + 255) / 256);
    DCM_LAUNCH(ctx, k_count<R>, nb, 256, 0, st, n, pos, grid, cell, ctx->slot, ctx->cell_count);
  }
  int rc = exclusive_scan(ctx, ctx->cell_count, cell_start, grid.ncell, st);
  if (rc) return rc;
  if (n > 0) {
    unsigned nb = (unsigned)((n + 255) / 256);
    launch_scatter(ctx, n, cell, ctx->slot, cell_start, perm, st);
    launch_cell_sort(ctx, grid.ncell, cell_start, perm, st);
    if (pos_sorted) k_gather<typename RT<R>::R4><<<nb, 256, 0, st>>>(n, perm, pos, pos_sorted);
  }
  return check_launch(ctx, "bin_particles");
}

template <typename R>
int histogram(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const Grid<R>& grid, int32_t* count,
              cudaStream_t st) {
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(count, 0, sizeof(int32_t) * grid.ncell, st));
  if (n > 0) DCM_LAUNCH(ctx, k_count<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, pos, grid, nullptr, nullptr, count);
  return check_launch(ctx, "histogram");
}

template int bin_particles<float>(dcm_ctx*, int64_t, const float4*, const Grid<float>&, int32_t*, int32_t*,
                                  int32_t*, float4*, cudaStream_t);
template int bin_particles<double>(dcm_ctx*, int64_t, const dvec4*, const Grid<double>&, int32_t*, int32_t*,
                                   int32_t*, dvec4*, cudaStream_t);
template int histogram<float>(dcm_ctx*, int64_t, const float4*, const Grid<float>&, int32_t*, cudaStream_t);
template int histogram<double>(dcm_ctx*, int64_t, const dvec4*, const Grid<double>&, int32_t*, cudaStream_t);

// Gather of a per-particle payload into sorted order (used by step.cu).
template <typename V>
void gather(dcm_ctx* ctx, int64_t n, const int32_t* perm, const V* src, V* dst, cudaStream_t st) {
  if (n > 0) DCM_LAUNCH(ctx, k_gather<V>, (unsigned)((n + 255) / 256), 256, 0, st, n, perm, src, dst);
}
template void gather<float4>(dcm_ctx*, int64_t, const int32_t*, const float4*, float4*, cudaStream_t);
template void gather<dvec4>(dcm_ctx*, int64_t, const int32_t*, const dvec4*, dvec4*, cudaStream_t);
template void gather<float>(dcm_ctx*, int64_t, const int32_t*, const float*, float*, cudaStream_t);
template void gather<double>(dcm_ctx*, int64_t, const int32_t*, const double*, double*, cudaStream_t);
template void gather<int32_t>(dcm_ctx*, int64_t, const int32_t*, const int32_t*, int32_t*, cudaStream_t);

// Scatter + per-cell stable sort for callers that computed cell and slot
// themselves (step.cu fuses the count into the drift kernel).
int scatter_sort(dcm_ctx* ctx, int64_t n, const int32_t* cell, const int32_t* slot, const int32_t* cell_start,
                 int64_t ncell, int32_t* perm, cudaStream_t st) {
  if (n > 0) {
    launch_scatter(ctx, n, cell, slot, cell_start, perm, st);
    launch_cell_sort(ctx, ncell, cell_start, perm, st);
  }
  return check_launch(ctx, "scatter_sort");
}

}  // namespace dcm
