// Removal of small connected components of the segmented volume S (Section
// 2.1: low-density "bubbles" in the high-density phase and vice versa are
// false detections and are filtered out by volume).  Components are sets of
// boxes of equal S joined through faces (6-connectivity, periodic); every
// component of fewer than params.min_component boxes takes the other value.
//
// Labelling: every box starts as its own tree (lab[b] = b).  A hook pass
// links, for each face between equal-valued boxes, the root of the larger
// tree index under the smaller one (atomicMin), a compress pass points every
// box straight at its root; the two alternate until a hook pass changes
// nothing.  The root of a component is then its smallest box index (no box
// of a component can ever point below it), so labels, sizes and the filtered
// volume do not depend on the order in which threads run.
#include <algorithm>

#include "dcm_internal.cuh"

namespace dcm {

constexpr int kCcPasses = 64;  // hook/compress passes before DCM_ERR_NOT_CONVERGED

// Root of b: parents only ever decrease (lab[b] <= b), so the walk ends; the
// bound only guards against a corrupted table.
__device__ __forceinline__ int32_t cc_root(const int32_t* lab, int32_t b) {
  for (int it = 0; it < (1 << 26); ++it) {
    int32_t p = lab[b];
    if (p == b) return b;
    b = p;
  }
  return b;
}

__global__ void k_cc_init(int64_t nbox, int32_t* __restrict__ lab, int32_t* __restrict__ flags) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbox) lab[b] = (int32_t)b;
  if (b < kCcPasses + 1) flags[b] = 0;
}

// Hook pass `pass`; skipped once an earlier pass changed nothing.
__global__ void k_cc_hook(const uint8_t* __restrict__ s, int nx, int ny, int nz, int32_t* lab, int32_t* flags,
                          int pass) {
  if (pass > 0 && flags[pass - 1] == 0) return;
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t nxy = (int64_t)nx * ny;
  if (b >= nxy * nz) return;
  int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / nxy);
  const uint8_t v = s[b];
  // the three forward faces cover every face once
  int64_t nb[3] = {(x + 1 == nx ? b - x : b + 1), (y + 1 == ny ? b - (int64_t)y * nx : b + nx),
                   (z + 1 == nz ? b - (int64_t)z * nxy : b + nxy)};
  bool changed = false;
  for (int k = 0; k < 3; ++k) {
    if (s[nb[k]] != v) continue;
    int32_t ra = cc_root(lab, (int32_t)b), rb = cc_root(lab, (int32_t)nb[k]);
    if (ra != rb) {
      atomicMin(lab + max(ra, rb), min(ra, rb));
      changed = true;
    }
  }
  if (changed) flags[pass] = 1;
}

__global__ void k_cc_compress(int64_t nbox, int32_t* lab, const int32_t* __restrict__ flags, int pass) {
  if (flags[pass] == 0) return;
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nbox) lab[b] = cc_root(lab, (int32_t)b);
}

// Component sizes at the roots (warp-aggregated: neighbouring boxes mostly
// share a root).  A hook pass that still changed something at the end of the
// budget raises DCM_ERR_NOT_CONVERGED.
__global__ void k_cc_count(int64_t nbox, const int32_t* __restrict__ lab, int32_t* __restrict__ cnt,
                           const int32_t* __restrict__ flags, int32_t* __restrict__ status) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0 && flags[kCcPasses - 1]) atomicCAS(status, 0, DCM_ERR_NOT_CONVERGED);
  bool ok = b < nbox;
  int32_t r = ok ? lab[b] : -1;
  unsigned peers = __match_any_sync(0xffffffffu, r);
  int lane = threadIdx.x & 31;
  if (ok && lane == __ffs(peers) - 1) atomicAdd(cnt + r, __popc(peers));
}

__global__ void k_cc_flip(int64_t nbox, const uint8_t* __restrict__ s_in, const int32_t* __restrict__ lab,
                          const int32_t* __restrict__ cnt, int32_t min_boxes, uint8_t* __restrict__ s_out) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  uint8_t v = s_in[b];
  s_out[b] = cnt[lab[b]] < min_boxes ? (uint8_t)(1 - v) : v;
}

// Liquid-side interface boxes of S (the rule of the segmentation kernel).
__global__ void k_interface_of(const uint8_t* __restrict__ s, int nx, int ny, int nz, uint8_t* __restrict__ iface) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t nxy = (int64_t)nx * ny;
  if (b >= nxy * nz) return;
  int x = (int)(b % nx), y = (int)((b / nx) % ny), z = (int)(b / nxy);
  int f = 0;
  if (s[b]) {
    f |= !s[x == 0 ? b + nx - 1 : b - 1];
    f |= !s[x == nx - 1 ? b - x : b + 1];
    f |= !s[y == 0 ? b + (int64_t)(ny - 1) * nx : b - nx];
    f |= !s[y == ny - 1 ? b - (int64_t)y * nx : b + nx];
    f |= !s[z == 0 ? b + (int64_t)(nz - 1) * nxy : b - nxy];
    f |= !s[z == nz - 1 ? b - (int64_t)z * nxy : b + nxy];
  }
  iface[b] = (uint8_t)f;
}

void interface_of(dcm_ctx* ctx, const uint8_t* s, uint8_t* iface, cudaStream_t st) {
  const int nx = (int)ctx->nh[0], ny = (int)ctx->nh[1], nz = (int)ctx->nh[2];
  DCM_LAUNCH(ctx, k_interface_of, (unsigned)((ctx->nbox + 255) / 256), 256, 0, st, s, nx, ny, nz, iface);
}

int remove_small_components(dcm_ctx* ctx, const uint8_t* s_in, uint8_t* s_out, uint8_t* iface, cudaStream_t st) {
  if (ctx->p.min_component <= 0 || !ctx->cc_lab)
    return set_error(ctx, DCM_ERR_INVALID_ARG, "the context was created with min_component = 0");
  int nx = (int)ctx->nh[0], ny = (int)ctx->nh[1], nz = (int)ctx->nh[2];
  int64_t nbox = ctx->nbox;
  if (nbox >= INT32_MAX) return set_error(ctx, DCM_ERR_CAPACITY, "component labels need < 2^31 boxes");
  unsigned nb = (unsigned)((std::max<int64_t>(nbox, kCcPasses + 1) + 255) / 256);
  DCM_LAUNCH(ctx, k_cc_init, nb, 256, 0, st, nbox, ctx->cc_lab, ctx->cc_flags);
  for (int pass = 0; pass < kCcPasses; ++pass) {
    DCM_LAUNCH(ctx, k_cc_hook, nb, 256, 0, st, s_in, nx, ny, nz, ctx->cc_lab, ctx->cc_flags, pass);
    DCM_LAUNCH(ctx, k_cc_compress, nb, 256, 0, st, nbox, ctx->cc_lab, ctx->cc_flags, pass);
  }
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cc_cnt, 0, sizeof(int32_t) * nbox, st));
  DCM_LAUNCH(ctx, k_cc_count, nb, 256, 0, st, nbox, ctx->cc_lab, ctx->cc_cnt, ctx->cc_flags, ctx->status);
  DCM_LAUNCH(ctx, k_cc_flip, nb, 256, 0, st, nbox, s_in, ctx->cc_lab, ctx->cc_cnt, ctx->p.min_component, s_out);
  DCM_LAUNCH(ctx, k_interface_of, nb, 256, 0, st, s_out, nx, ny, nz, iface);
  return check_launch(ctx, "remove_small_components");
}

}  // namespace dcm
