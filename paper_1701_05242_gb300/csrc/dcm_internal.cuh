// Internal declarations shared by the CUDA translation units of libdcm.
// Not part of the public ABI (see include/dcm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>

#include "../../include/dcm.h"

namespace dcm {

// ----------------------------------------------------------------------------
// Precision traits.  The mixed form stores float4 / float, the FP64 form a
// 32-byte aligned 4-vector of doubles (CUDA 13 deprecates double4).
// ----------------------------------------------------------------------------
struct __align__(32) dvec4 {
  double x, y, z, w;
};

template <typename R>
struct RT;
template <>
struct RT<float> {
  using R4 = float4;
  __device__ static float inf() { return __int_as_float(0x7f800000); }
};
template <>
struct RT<double> {
  using R4 = dvec4;
  __device__ static double inf() { return __longlong_as_double(0x7ff0000000000000LL); }
};

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ dvec4 ldg4(const dvec4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return dvec4{a.x, a.y, b.x, b.y};
}

// Exact floor(x / l) for an edge l with a short mantissa (k * l exact), clamped
// to [0, n-1].  One correction step suffices because x * (1/l) is within one
// unit of the true quotient.  The quotient is first clamped to [-1, n] (NaN
// to -1), so that coordinates far outside the box stay clear of integer
// overflow.
template <typename R>
__device__ __forceinline__ int cell_coord(R x, R l, R inv_l, int n) {
  R q = fmin(fmax(floor(x * inv_l), (R)-1), (R)n);
  int k = (int)q;
  if ((R)k * l > x)
    --k;
  else if ((R)(k + 1) * l <= x)
    ++k;
  k = k < 0 ? 0 : k;
  return k > n - 1 ? n - 1 : k;
}

// ----------------------------------------------------------------------------
// Geometry handed to kernels by value.
// ----------------------------------------------------------------------------
template <typename R>
struct Grid {
  int n[3];      // cells per dimension
  R edge;        // cell edge along y and z
  R inv_edge;
  R edge_x;      // cell edge along x, the direction of the contiguous cell rows
  R inv_edge_x;
  R L[3];        // box lengths (= n * edge exactly)
  int64_t ncell;
};

struct LJTable {
  int ntypes;
  float eps24[16], eps4[16], sig2[16];   // FP32 copies
  double deps24[16], deps4[16], dsig2[16];
};

// ----------------------------------------------------------------------------
// Context.
// ----------------------------------------------------------------------------
}  // namespace dcm

struct dcm_ctx {
  dcm_params p;
  int precision;
  int64_t nc[3], ncell;     // force cells
  int64_t nh[3], nbox;      // density boxes
  int64_t n_max;
  int device;
  char err[512];
  // device scratch
  int32_t* status;          // [4]: first device-side error code, ...
  uint32_t* coop_sync;      // [4]: grid-barrier words of the cooperative distance sweeps
  int32_t* slot;            // n_max: rank of a particle inside its cell (atomics)
  int32_t* cell;            // n_max: cell of each particle (step)
  int32_t* perm;            // n_max
  int32_t* cell_start;      // ncell + 1
  int32_t* cell_count;      // ncell
  unsigned long long* scan_state;  // [scan_cap + 1]: look-back words of the scan tiles, ticket
  int32_t* box_count;       // nbox
  int32_t* g;               // nbox
  int32_t* g_tmp;           // nbox
  uint8_t* s;               // nbox
  uint8_t* iface;           // nbox
  void* D[2];               // nbox reals each
  int32_t* flags;           // iter_max + 2 change flags of the distance sweeps
  int32_t* hist;            // histogram of box sums
  int32_t* thr;             // [8]: gmin, gmax, T, sweeps, ...
  double* red;              // reduction partials
  double* red_tmp;          // [8 * 256] first-level chunk sums
  double* adj_part;         // [32][red_cap] adjoint parameter-gradient partials
  double* adj_pairs;        // [48]: per-pair eps sums, per-pair sigma sums, eps values
  double* totals;           // [4]
  int32_t* host_status;     // pinned host mirror
  int64_t red_cap;          // number of partial slots in red (per quantity)
  int32_t* blk_max;         // nblk: largest cutoff (float bits) per adjoint block
  int32_t* tile_scratch;    // tile_scratch_ints(n_max): launch order of the force and adjoint tiles
  int nblk3[3];             // adjoint blocks per dimension (edge >= 1.001 rc_max)
  int64_t nblk;
  int64_t scan_cap;
  int64_t launches;         // kernels launched through this context
  // Verlet lists (params.skin > 0)
  int32_t* nnb;             // n_max: same-image entries of each list (from the front)
  int32_t* nimg;            // n_max: periodic-image entries of each list (from the back)
  // distance sweeps: queues of boxes to re-solve, their lengths per sweep,
  // the last sweep each box was queued for, and the boxes fixed at 0
  int32_t* dq[2];
  int32_t* dqlen;
  int32_t* dstamp;
  uint8_t* dfixed;
  // bubble filter (params.min_component > 0)
  int32_t* cc_lab;          // nbox: component tree parents
  int32_t* cc_cnt;          // nbox: component sizes at the roots
  int32_t* cc_flags;        // hook passes that changed a parent
  uint8_t* cc_s0;           // nbox: S before the filter
  int32_t* capw;            // per warp: longest list of its 32 particles
  int32_t* offw;            // exclusive scan of capw (units of 32 entries)
  uint32_t* list;           // interleaved lists (grown on demand)
  int64_t list_cap;
  void* xbuild;             // positions at the last build
  int32_t* dmax;            // largest squared displacement (float bits)
  int32_t* lflag;           // list overflow flag of the single-walk build
  int list_valid;
  // regularised segmentation (params.segmentation = 1)
  void* ms_u;               // nbox reals: relaxed volume u
  void* ms_ub;              // nbox reals: extrapolated u
  void* ms_p;               // 3 nbox reals: dual value per face
  void* ms_w;               // nbox reals: data weights
  unsigned long long* ms_sums;  // [ms_outer][4]: n0, S0, n1, S1
  double* ms_c;             // [2]: phase values of the last outer iteration
  int32_t* ms_flags;        // [ms_outer + 2]: stop mark, then "changed" per outer iteration
  // optional per-stage CUDA-event timing (dcm_set_timing)
  int timing;
  int ev_n[DCM_NSTAGES];
  int ev_cap;                        // event pairs per stage
  cudaEvent_t* ev;                   // [DCM_NSTAGES][ev_cap][2]
};

namespace dcm {

constexpr int kHistCap = 1 << 20;
constexpr int kScanBlock = 512;        // threads of the scan kernel (two blocks per SM at its registers)
constexpr int kScanItems = 16;         // items per thread (four 16-byte loads)
constexpr int kScanTile = kScanBlock * kScanItems;
// Launch order of tiles (the particles of one block) by decreasing cost key
// (tile_order.cu): a stable counting sort over kTileBins bins, chunks of
// kTileChunk tiles.  Scratch: order[ntile], key[ntile], the bin counts of
// every chunk [kTileBins][nchunk].
constexpr int kTileBins = 64;
constexpr int kTileChunk = 1024;
constexpr int64_t tile_chunks(int64_t ntile) { return (ntile + kTileChunk - 1) / kTileChunk; }
constexpr int64_t tile_order_ints(int64_t ntile) { return 2 * ntile + kTileBins * tile_chunks(ntile) + 1; }
// tiles of at least 32 particles
constexpr int64_t tile_scratch_ints(int64_t n_max) { return tile_order_ints((n_max + 31) / 32 + 1); }

int set_error(dcm_ctx* ctx, int code, const char* fmt, ...);

// Cell-list force kernel and per-particle accumulation form of a context.
int scan_wait_selftest(dcm_ctx* ctx, cudaStream_t st);  // the look-back scan's bounded wait
int force_kernel_choice(const dcm_params& p);  // DCM_FORCE_* with AUTO resolved
int resolve_force_kernel(const dcm_ctx* ctx);  // ... and each kernel's limits applied
int resolve_accumulation(const dcm_ctx* ctx);  // DCM_ACC_* that the force launches run

// Stage timing: events recorded on the launching stream around a stage.
void stage_begin(dcm_ctx* ctx, int stage, cudaStream_t st);
void stage_end(dcm_ctx* ctx, int stage, cudaStream_t st);
int check_launch(dcm_ctx* ctx, const char* what);

// Grids from the context.
template <typename R>
Grid<R> cell_grid(const dcm_ctx* ctx);
template <typename R>
Grid<R> box_grid(const dcm_ctx* ctx);
LJTable lj_table(const dcm_params& p);
// The one-type kernels take eps = sigma = 1 as constants; anything else uses
// the per-pair parameter path.
inline bool lj_general(const LJTable& t) {
  return t.ntypes > 1 || t.deps24[0] != 24.0 || t.dsig2[0] != 1.0;
}

// ---- launchers (one per translation unit) ----------------------------------
// bin.cu
template <typename R>
int bin_particles(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const Grid<R>& grid,
                  int32_t* cell, int32_t* cell_start, int32_t* perm, typename RT<R>::R4* pos_sorted,
                  cudaStream_t st);
template <typename R>
int histogram(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const Grid<R>& grid,
              int32_t* count, cudaStream_t st);
int exclusive_scan(dcm_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);
template <typename V>
void gather(dcm_ctx* ctx, int64_t n, const int32_t* perm, const V* src, V* dst, cudaStream_t st);
int scatter_sort(dcm_ctx* ctx, int64_t n, const int32_t* cell, const int32_t* slot, const int32_t* cell_start,
                 int64_t ncell, int32_t* perm, cudaStream_t st);

// detect.cu
// Section 2.1's bubble filter on S (params.min_component > 0): s_out and the
// interface boxes of s_out (components.cu).
int remove_small_components(dcm_ctx* ctx, const uint8_t* s_in, uint8_t* s_out, uint8_t* iface, cudaStream_t st);
int detect_interface(dcm_ctx* ctx, const int32_t* box_count, uint8_t* s, uint8_t* iface,
                     int32_t* threshold, int32_t* g_out, cudaStream_t st);
// segment_ms.cu: the regularised two-phase segmentation of the box counts,
// refining s in place (params.segmentation = 1).
int ms_segment(dcm_ctx* ctx, const int32_t* count, uint8_t* s, cudaStream_t st);
// components.cu: interface boxes of a segmented volume.
void interface_of(dcm_ctx* ctx, const uint8_t* s, uint8_t* iface, cudaStream_t st);

// distance.cu
template <typename R>
int distance_sweeps(dcm_ctx* ctx, const uint8_t* s, const uint8_t* iface, R* D, int32_t* iters,
                    bool host_check, cudaStream_t st);

// cutoffs.cu
template <typename R>
int assign_cutoffs(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* D, R* rc,
                   cudaStream_t st);

// forces.cu.  energies = false (and no totals): the packed kernel sums the
// forces only (the force's w, the per-particle energy, is then zero), for
// the timesteps of dcm_step whose energy and virial nothing reads.
template <typename R>
int lj_forces(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc,
              const int32_t* cell_start, typename RT<R>::R4* force, double* totals, cudaStream_t st,
              bool energies = true);

// adjoint.cu
template <typename R>
int lj_adjoint(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc, const int32_t* cell_start,
               const typename RT<R>::R4* A, double dlde, typename RT<R>::R4* G, double* dparams, cudaStream_t st);

// verlet.cu
template <typename R>
int list_build(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc, cudaStream_t st);
// energies: whether the caller reads energy and virial (the list kernels sum
// them in any case).
template <typename R>
int list_forces(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc, typename RT<R>::R4* force,
                double* totals, cudaStream_t st, bool energies = true);
template <typename R>
int list_kick_drift(dcm_ctx* ctx, dcm_state* s, int64_t n, R hdt, R dt, int kicks, bool* rebuild, cudaStream_t st);
template <typename R>
int list_wrap_count(dcm_ctx* ctx, dcm_state* s, int64_t n, cudaStream_t st);

// step.cu
template <typename R>
int step_init(dcm_ctx* ctx, dcm_state* st, int64_t n, cudaStream_t stream);
template <typename R>
int step_run(dcm_ctx* ctx, dcm_state* st, int64_t n, double dt, int nsteps, cudaStream_t stream);

// Deterministic reduction of per-block partials (nblk x nq doubles, quantity-
// major) into out[0..nq) (device), optionally adding.  reduce.cu
int reduce_partials(dcm_ctx* ctx, const double* part, int64_t nblk, int nq, double* out, bool accumulate,
                    cudaStream_t st);

// Device status word: first error wins.
__device__ __forceinline__ void raise_status(int32_t* status, int code) { atomicCAS(status, 0, code); }

}  // namespace dcm

// Launch a kernel and count it.
#define DCM_LAUNCH(ctx, kernel, grid, block, smem, stream, ...)          \
  do {                                                                  \
    ++(ctx)->launches;                                                  \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);         \
  } while (0)

#define DCM_CUDA_TRY(ctx, call)                                                              \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return ::dcm::set_error((ctx), DCM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
