// C ABI of libdcm: parameter validation, context and scratch management, and
// dispatch of the public calls to the precision-specific launchers.
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <new>

#include "dcm_internal.cuh"

namespace dcm {

int set_error(dcm_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

int force_kernel_choice(const dcm_params& p) {
  return p.force_kernel == DCM_FORCE_AUTO ? DCM_FORCE_PACKED : p.force_kernel;
}

int check_launch(dcm_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(ctx, DCM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return DCM_OK;
}

template <typename R>
static Grid<R> make_grid(const int64_t* n, double edge, double edge_x, const double* box) {
  Grid<R> g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = (int)n[d];
    g.L[d] = (R)((double)n[d] * (d == 0 ? edge_x : edge));  // exact: short-mantissa edge times a small integer
  }
  g.edge = (R)edge;
  g.inv_edge = (R)(1.0 / edge);
  g.edge_x = (R)edge_x;
  g.inv_edge_x = (R)(1.0 / edge_x);
  g.ncell = n[0] * n[1] * n[2];
  (void)box;
  return g;
}

template <typename R>
Grid<R> cell_grid(const dcm_ctx* ctx) {
  return make_grid<R>(ctx->nc, ctx->p.l, ctx->p.lx, ctx->p.box);
}
template <typename R>
Grid<R> box_grid(const dcm_ctx* ctx) {
  return make_grid<R>(ctx->nh, ctx->p.h, ctx->p.h, ctx->p.box);
}
template Grid<float> cell_grid<float>(const dcm_ctx*);
template Grid<double> cell_grid<double>(const dcm_ctx*);
template Grid<float> box_grid<float>(const dcm_ctx*);
template Grid<double> box_grid<double>(const dcm_ctx*);

// Lorentz-Berthelot mixing: eps_ab = sqrt(eps_a eps_b), sigma_ab = (sigma_a + sigma_b) / 2.
LJTable lj_table(const dcm_params& p) {
  LJTable t;
  memset(&t, 0, sizeof(t));
  t.ntypes = p.ntypes;
  for (int a = 0; a < p.ntypes; ++a)
    for (int b = 0; b < p.ntypes; ++b) {
      double e = std::sqrt(p.eps[a] * p.eps[b]);
      double s = 0.5 * (p.sigma[a] + p.sigma[b]);
      int k = a * p.ntypes + b;
      t.deps24[k] = 24.0 * e;
      t.deps4[k] = 4.0 * e;
      t.dsig2[k] = s * s;
      t.eps24[k] = (float)t.deps24[k];
      t.eps4[k] = (float)t.deps4[k];
      t.sig2[k] = (float)t.dsig2[k];
    }
  return t;
}

static cudaEvent_t& event_at(dcm_ctx* ctx, int stage, int k, int e) {
  return ctx->ev[((int64_t)stage * ctx->ev_cap + k) * 2 + e];
}

void stage_begin(dcm_ctx* ctx, int stage, cudaStream_t st) {
  if (!ctx->timing) return;
  int k = ctx->ev_n[stage];
  if (k < ctx->ev_cap) cudaEventRecord(event_at(ctx, stage, k, 0), st);
}

void stage_end(dcm_ctx* ctx, int stage, cudaStream_t st) {
  if (!ctx->timing) return;
  int k = ctx->ev_n[stage];
  if (k < ctx->ev_cap) cudaEventRecord(event_at(ctx, stage, k, 1), st);
  ctx->ev_n[stage] = k + 1;
}

}  // namespace dcm

using namespace dcm;

// ---------------------------------------------------------------------------
// host-only helpers
// ---------------------------------------------------------------------------
static int msg_out(char* msg, int32_t len, int code, const char* fmt, ...) {
  if (msg && len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, (size_t)len, fmt, ap);
    va_end(ap);
  }
  return code;
}

// edge has at most 8 significant bits: edge * 2^m is an integer below 256 for some m
static bool short_mantissa(double v) {
  if (!(v > 0.0) || !std::isfinite(v)) return false;
  for (int m = -40; m <= 40; ++m) {
    double x = std::ldexp(v, m);
    if (x >= 256.0) return false;
    if (x >= 1.0 && x == std::floor(x)) return true;
  }
  return false;
}

static bool grid_of(double L, double edge, int64_t* n) {
  double q = L / edge;
  int64_t k = (int64_t)std::llround(q);
  if (k < 1 || std::fabs((double)k * edge - L) > 1e-9 * L) return false;
  *n = k;
  return true;
}

extern "C" int dcm_params_default(dcm_params* p) {
  if (!p) return DCM_ERR_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  p->h = 1.5;
  p->l = 1.5;
  p->rc_min = 3.0;
  p->rc_max = 6.0;
  p->ramp = 0.0;
  p->r_grid = 0.0;
  p->smooth_w = 2;
  p->threshold = -1;
  p->iter_max = 1000;
  p->ntypes = 1;
  for (int k = 0; k < 4; ++k) {
    p->eps[k] = 1.0;
    p->sigma[k] = 1.0;
  }
  p->shift_energy = 0;
  p->precision = DCM_PREC_MIXED;
  p->recompute_every = 10;
  p->n_max = 0;
  p->ms_inner = 200;
  p->ms_outer = 4;
  p->ms_nu = 4.0;
  return DCM_OK;
}

// Blocks of the adjoint's reverse-pair bound along axis d: edge at least
// 1.001 rc_max, so that any particle within rc_max of another lies in one of
// the 27 blocks around it even after the rounding of the block index.
static int64_t adjoint_blocks(const dcm_params* p, int d) {
  int64_t k = (int64_t)std::floor(p->box[d] / (1.001 * p->rc_max));
  return k < 1 ? 1 : k;
}

// Cell edge along axis d: lx along x when it is set, l otherwise.
static double cell_edge(const dcm_params* p, int d) { return d == 0 && p->lx > 0.0 ? p->lx : p->l; }

// Resolve the defaults that depend on other fields.
static dcm_params resolved(const dcm_params* p) {
  dcm_params q = *p;
  if (!(q.lx > 0.0)) q.lx = q.l;
  if (!(q.ramp > 0.0)) q.ramp = q.rc_max - q.rc_min;
  if (!(q.r_grid > 0.0)) q.r_grid = q.ramp + 2.0 * q.h;
  return q;
}

extern "C" int dcm_validate_params(const dcm_params* p, char* msg, int32_t len) {
  if (!p) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "params is NULL");
  if (msg && len > 0) msg[0] = 0;
  for (int d = 0; d < 3; ++d)
    if (!(p->box[d] > 0.0) || !std::isfinite(p->box[d]))
      return msg_out(msg, len, DCM_ERR_BOX, "box[%d] = %g must be positive", d, p->box[d]);
  if (!short_mantissa(p->l)) return msg_out(msg, len, DCM_ERR_BOX, "cell edge l = %g needs a short mantissa", p->l);
  if (!short_mantissa(p->h)) return msg_out(msg, len, DCM_ERR_BOX, "box edge h = %g needs a short mantissa", p->h);
  if (!(p->lx >= 0.0) || !std::isfinite(p->lx))
    return msg_out(msg, len, DCM_ERR_INVALID_ARG, "lx = %g must be >= 0 (0: l)", p->lx);
  if (p->lx > 0.0 && !short_mantissa(p->lx))
    return msg_out(msg, len, DCM_ERR_BOX, "cell edge lx = %g needs a short mantissa", p->lx);
  int64_t n;
  for (int d = 0; d < 3; ++d) {
    if (!grid_of(p->box[d], cell_edge(p, d), &n) || n >= 65536)
      return msg_out(msg, len, DCM_ERR_BOX, "box[%d] = %g is not a multiple of the cell edge %g (below 65536 cells)",
                     d, p->box[d], cell_edge(p, d));
    if (!grid_of(p->box[d], p->h, &n) || n >= 65536)
      return msg_out(msg, len, DCM_ERR_BOX, "box[%d] = %g is not a multiple of h = %g (below 65536 boxes)", d,
                     p->box[d], p->h);
  }
  if (!(p->rc_min > 0.0) || !(p->rc_max >= p->rc_min))
    return msg_out(msg, len, DCM_ERR_INVALID_ARG, "need 0 < rc_min <= rc_max (got %g, %g)", p->rc_min, p->rc_max);
  double Lmin = std::fmin(p->box[0], std::fmin(p->box[1], p->box[2]));
  if (p->rc_max > 0.5 * Lmin)
    return msg_out(msg, len, DCM_ERR_BOX, "rc_max = %g exceeds half the smallest box length %g", p->rc_max, Lmin);
  if (p->ntypes < 1 || p->ntypes > 4)
    return msg_out(msg, len, DCM_ERR_INVALID_ARG, "ntypes = %d not in 1..4", p->ntypes);
  for (int k = 0; k < p->ntypes; ++k)
    if (!(p->eps[k] > 0.0) || !(p->sigma[k] > 0.0))
      return msg_out(msg, len, DCM_ERR_INVALID_ARG, "eps/sigma of type %d must be positive", k);
  if (p->smooth_w < 0) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "smooth_w must be >= 0");
  if (p->iter_max < 1 || p->iter_max > 100000)
    return msg_out(msg, len, DCM_ERR_INVALID_ARG, "iter_max must be in 1..100000");
  if (p->recompute_every < 1) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "recompute_every must be >= 1");
  if (p->min_component < 0) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "min_component must be >= 0");
  if (p->force_kernel != DCM_FORCE_AUTO && p->force_kernel != DCM_FORCE_THREAD && p->force_kernel != DCM_FORCE_PACKED)
    return msg_out(msg, len, DCM_ERR_INVALID_ARG, "force_kernel must be one of DCM_FORCE_*");
  if (p->accumulation < DCM_ACC_AUTO || p->accumulation > DCM_ACC_PLANE_KAHAN)
    return msg_out(msg, len, DCM_ERR_INVALID_ARG, "accumulation must be one of DCM_ACC_*");
  if (p->newton3 != 0 && p->newton3 != 1) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "newton3 must be 0 or 1");
  if (p->segmentation != 0 && p->segmentation != 1)
    return msg_out(msg, len, DCM_ERR_INVALID_ARG, "segmentation must be 0 or 1");
  if (p->segmentation) {
    if (!(p->ms_nu >= 0.0) || !std::isfinite(p->ms_nu))
      return msg_out(msg, len, DCM_ERR_INVALID_ARG, "ms_nu must be finite and >= 0");
    if (p->ms_inner < 1 || p->ms_inner > 100000) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "ms_inner in 1..100000");
    if (p->ms_outer < 1 || p->ms_outer > 64) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "ms_outer in 1..64");
  }
  if (p->newton3 && !(p->skin > 0.0))
    return msg_out(msg, len, DCM_ERR_INVALID_ARG, "newton3 needs Verlet lists (skin > 0)");
  if (p->precision != DCM_PREC_FP64 && p->precision != DCM_PREC_MIXED)
    return msg_out(msg, len, DCM_ERR_INVALID_ARG, "precision must be DCM_PREC_FP64 or DCM_PREC_MIXED");
  if (p->n_max < 0 || p->n_max > 0x7fffffffLL) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "n_max out of range");
  int64_t nc[3], nh[3];
  for (int d = 0; d < 3; ++d) {
    grid_of(p->box[d], cell_edge(p, d), nc + d);
    grid_of(p->box[d], p->h, nh + d);
  }
  if (nc[0] * nc[1] * nc[2] >= 0x7fffffffLL || nh[0] * nh[1] * nh[2] >= 0x7fffffffLL)
    return msg_out(msg, len, DCM_ERR_BOX, "grid too large for 32-bit cell indices");
  dcm_params q = resolved(p);
  if (!(q.r_grid > 0.0)) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "r_grid must be positive");
  if (!(p->skin >= 0.0) || !std::isfinite(p->skin)) return msg_out(msg, len, DCM_ERR_INVALID_ARG, "skin must be >= 0");
  if (p->skin > 0.0) {
    if (p->rc_max + p->skin > 0.5 * Lmin)
      return msg_out(msg, len, DCM_ERR_BOX, "rc_max + skin = %g exceeds half the smallest box length %g",
                     p->rc_max + p->skin, Lmin);
    if (p->n_max >= (int64_t)1 << 26) return msg_out(msg, len, DCM_ERR_CAPACITY, "Verlet lists need n_max < 2^26");
  }
  return DCM_OK;
}

extern "C" int dcm_grid_dims(const dcm_params* p, int64_t* cells3, int64_t* boxes3) {
  if (dcm_validate_params(p, nullptr, 0) != DCM_OK) return DCM_ERR_BOX;
  for (int d = 0; d < 3; ++d) {
    if (cells3) grid_of(p->box[d], cell_edge(p, d), cells3 + d);
    if (boxes3) grid_of(p->box[d], p->h, boxes3 + d);
  }
  return DCM_OK;
}

struct ScratchPlan {
  int64_t n_max, ncell, nbox, scan_cap, red_cap, rsize, flags, nblk;
  double skin;
  int32_t min_component, segmentation, ms_outer;
  int64_t total() const {
    return 4 * 4 + 16 + 3 * 4 * n_max + 4 * (ncell + 1) + 4 * ncell + 8 * (scan_cap + 1) + 3 * 4 * nbox + 2 * nbox +
           2 * rsize * nbox + 4 * flags + 4 * (int64_t)kHistCap + 4 * 8 + 8 * 3 * red_cap + 8 * 8 + 8 * 8 * 256 +
           8 * 32 * red_cap + 8 * 48 + (skin > 0 ? 8 * n_max + 8 * (n_max / 32 + 16) + 4 * rsize * n_max + 32 : 0) +
           (min_component > 0 ? 9 * nbox + 4 * 80 : 0) + 13 * nbox + 4 * (flags + 2) + 4 * nblk +
           4 * tile_scratch_ints(n_max) +
           (segmentation ? 6 * rsize * nbox + 32 * ms_outer + 16 + 4 * (ms_outer + 2) : 0);
  }
};

static ScratchPlan plan_of(const dcm_params* p) {
  ScratchPlan s;
  int64_t nc[3], nh[3];
  for (int d = 0; d < 3; ++d) {
    grid_of(p->box[d], cell_edge(p, d), nc + d);
    grid_of(p->box[d], p->h, nh + d);
  }
  s.n_max = p->n_max;
  s.ncell = nc[0] * nc[1] * nc[2];
  s.nbox = nh[0] * nh[1] * nh[2];
  int64_t big = s.ncell > s.nbox ? s.ncell : s.nbox;
  s.scan_cap = (big + kScanTile - 1) / kScanTile + 1;
  s.red_cap = ((s.n_max + 255) / 256 + 1) * 8;  // one partial per warp of the padded launches
  s.rsize = p->precision == DCM_PREC_FP64 ? 8 : 4;
  s.flags = p->iter_max + 2;
  s.skin = p->skin;
  s.min_component = p->min_component;
  s.segmentation = p->segmentation;
  s.ms_outer = p->ms_outer;
  s.nblk = adjoint_blocks(p, 0) * adjoint_blocks(p, 1) * adjoint_blocks(p, 2);
  return s;
}

extern "C" int dcm_scratch_bytes(const dcm_params* p, int64_t* bytes) {
  if (!bytes) return DCM_ERR_INVALID_ARG;
  int r = dcm_validate_params(p, nullptr, 0);
  if (r) return r;
  *bytes = plan_of(p).total();
  return DCM_OK;
}

extern "C" const char* dcm_version(void) { return "dcm-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" void dcm_destroy(dcm_ctx* ctx) {
  if (!ctx) return;
  void* dev[] = {ctx->status, ctx->coop_sync, ctx->slot,  ctx->cell,  ctx->perm,  ctx->cell_start, ctx->cell_count,
                 ctx->scan_state, ctx->box_count, ctx->g, ctx->g_tmp, ctx->s, ctx->iface,
                 ctx->D[1], ctx->flags, ctx->hist, ctx->thr, ctx->red, ctx->totals, ctx->D[0], ctx->red_tmp, ctx->adj_part, ctx->adj_pairs,
                 ctx->nnb, ctx->nimg, ctx->capw, ctx->offw, ctx->list, ctx->xbuild, ctx->dmax, ctx->lflag,
                 ctx->cc_lab, ctx->cc_cnt, ctx->cc_flags, ctx->cc_s0, ctx->dq[0], ctx->dq[1], ctx->dqlen,
                 ctx->dstamp, ctx->dfixed, ctx->blk_max, ctx->tile_scratch, ctx->ms_u, ctx->ms_ub, ctx->ms_p, ctx->ms_w,
                 ctx->ms_sums, ctx->ms_c, ctx->ms_flags};
  for (void* q : dev)
    if (q) cudaFree(q);
  if (ctx->host_status) cudaFreeHost(ctx->host_status);
  if (ctx->ev) {
    for (int64_t k = 0; k < (int64_t)DCM_NSTAGES * ctx->ev_cap * 2; ++k)
      if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    free(ctx->ev);
  }
  delete ctx;
}

extern "C" int dcm_create(const dcm_params* p, dcm_ctx** out) {
  if (!out) return DCM_ERR_INVALID_ARG;
  *out = nullptr;
  int r = dcm_validate_params(p, nullptr, 0);
  if (r) return r;
  dcm_ctx* ctx = new (std::nothrow) dcm_ctx();
  if (!ctx) return DCM_ERR_NOMEM;
  memset(ctx, 0, sizeof(*ctx));
  ctx->p = resolved(p);
  ctx->precision = p->precision;
  for (int d = 0; d < 3; ++d) {
    grid_of(p->box[d], cell_edge(p, d), ctx->nc + d);
    grid_of(p->box[d], p->h, ctx->nh + d);
    ctx->p.box[d] = (double)ctx->nc[d] * cell_edge(p, d);  // exact multiple of the cell edge
  }
  ctx->ncell = ctx->nc[0] * ctx->nc[1] * ctx->nc[2];
  ctx->nbox = ctx->nh[0] * ctx->nh[1] * ctx->nh[2];
  ctx->n_max = p->n_max;
  cudaGetDevice(&ctx->device);
  ScratchPlan s = plan_of(p);
  ctx->scan_cap = s.scan_cap;
  ctx->red_cap = s.red_cap;
  int64_t nm = s.n_max > 0 ? s.n_max : 1;
  bool ok = true;
  auto alloc = [&](void** ptr, int64_t bytes) {
    if (!ok) return;
    if (cudaMalloc(ptr, (size_t)(bytes > 0 ? bytes : 16)) != cudaSuccess) ok = false;
  };
  alloc((void**)&ctx->status, 16);
  alloc((void**)&ctx->coop_sync, 16);
  alloc((void**)&ctx->slot, 4 * nm);
  alloc((void**)&ctx->cell, 4 * nm);
  alloc((void**)&ctx->perm, 4 * nm);
  alloc((void**)&ctx->cell_start, 4 * (s.ncell + 1));
  alloc((void**)&ctx->cell_count, 4 * s.ncell);
  alloc((void**)&ctx->scan_state, 8 * (s.scan_cap + 1));
  alloc((void**)&ctx->box_count, 4 * s.nbox);
  alloc((void**)&ctx->g, 4 * s.nbox);
  alloc((void**)&ctx->g_tmp, 4 * s.nbox);
  alloc((void**)&ctx->s, s.nbox);
  alloc((void**)&ctx->iface, s.nbox);
  alloc(&ctx->D[0], s.rsize * s.nbox);
  alloc(&ctx->D[1], s.rsize * s.nbox);
  alloc((void**)&ctx->flags, 4 * s.flags);
  alloc((void**)&ctx->hist, 4 * (int64_t)kHistCap);
  alloc((void**)&ctx->thr, 4 * 8);
  alloc((void**)&ctx->red, 8 * 3 * s.red_cap);
  alloc((void**)&ctx->totals, 8 * 8);
  alloc((void**)&ctx->red_tmp, 8 * 8 * 256);
  alloc((void**)&ctx->adj_part, 8 * 32 * s.red_cap);
  if (p->skin > 0.0) {
    alloc((void**)&ctx->nnb, 4 * nm);
    alloc((void**)&ctx->nimg, 4 * nm);
    alloc((void**)&ctx->capw, 4 * (nm / 32 + 16));
    alloc((void**)&ctx->offw, 4 * (nm / 32 + 16));
    alloc(&ctx->xbuild, 4 * s.rsize * nm);
    alloc((void**)&ctx->dmax, 16);
    alloc((void**)&ctx->lflag, 16);
  }
  alloc((void**)&ctx->dq[0], 4 * s.nbox);
  alloc((void**)&ctx->dq[1], 4 * s.nbox);
  alloc((void**)&ctx->dqlen, 4 * (int64_t)(p->iter_max + 2));
  alloc((void**)&ctx->dstamp, 4 * s.nbox);
  alloc((void**)&ctx->dfixed, s.nbox);
  if (p->min_component > 0) {
    alloc((void**)&ctx->cc_lab, 4 * s.nbox);
    alloc((void**)&ctx->cc_cnt, 4 * s.nbox);
    alloc((void**)&ctx->cc_flags, 4 * 80);
    alloc((void**)&ctx->cc_s0, s.nbox);
  }
  if (p->segmentation) {
    alloc(&ctx->ms_u, s.rsize * s.nbox);
    alloc(&ctx->ms_ub, s.rsize * s.nbox);
    alloc(&ctx->ms_p, 3 * s.rsize * s.nbox);
    alloc(&ctx->ms_w, s.rsize * s.nbox);
    alloc((void**)&ctx->ms_sums, 32 * (int64_t)p->ms_outer);
    alloc((void**)&ctx->ms_c, 16);
    alloc((void**)&ctx->ms_flags, 4 * (int64_t)(p->ms_outer + 2));
  }
  alloc((void**)&ctx->adj_pairs, 8 * 48);
  for (int d = 0; d < 3; ++d) ctx->nblk3[d] = (int)adjoint_blocks(p, d);  // as counted in the plan
  ctx->nblk = s.nblk;
  alloc((void**)&ctx->blk_max, 4 * s.nblk);
  alloc((void**)&ctx->tile_scratch, 4 * tile_scratch_ints(s.n_max));
  if (ok && cudaMallocHost((void**)&ctx->host_status, 16) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    dcm_destroy(ctx);
    return DCM_ERR_NOMEM;
  }
  if (cudaMemset(ctx->status, 0, 16) != cudaSuccess || cudaMemset(ctx->totals, 0, 64) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    dcm_destroy(ctx);
    return DCM_ERR_CUDA;
  }
  *out = ctx;
  return DCM_OK;
}

extern "C" const char* dcm_last_error(const dcm_ctx* ctx) { return ctx ? ctx->err : "null context"; }

extern "C" int dcm_status(dcm_ctx* ctx, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  DCM_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->host_status, ctx->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  DCM_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  int code = ctx->host_status[0];
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int32_t), st));
  if (code) set_error(ctx, code, "device status %d", code);
  return code;
}

extern "C" int dcm_scan_wait_selftest(dcm_ctx* ctx, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  int r = scan_wait_selftest(ctx, (cudaStream_t)stream);
  if (r) return r;
  return dcm_status(ctx, stream);
}

// ---------------------------------------------------------------------------
// hot path
// ---------------------------------------------------------------------------
#define REQUIRE(cond, ...)                                                  \
  do {                                                                      \
    if (!(cond)) return set_error(ctx, DCM_ERR_INVALID_ARG, __VA_ARGS__);   \
  } while (0)

static int check_n(dcm_ctx* ctx, int64_t n) {
  if (n < 0) return set_error(ctx, DCM_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
  if (n > ctx->n_max)
    return set_error(ctx, DCM_ERR_CAPACITY, "n = %lld exceeds n_max = %lld", (long long)n, (long long)ctx->n_max);
  return DCM_OK;
}

extern "C" int dcm_bin(dcm_ctx* ctx, int64_t n, const void* pos, int32_t* cell, int32_t* cell_start, int32_t* perm,
                       void* pos_sorted, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  int r = check_n(ctx, n);
  if (r) return r;
  REQUIRE(cell_start && (n == 0 || (pos && cell && perm)), "dcm_bin: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->precision == DCM_PREC_MIXED)
    return bin_particles<float>(ctx, n, (const float4*)pos, cell_grid<float>(ctx), cell, cell_start, perm,
                                (float4*)pos_sorted, st);
  return bin_particles<double>(ctx, n, (const dvec4*)pos, cell_grid<double>(ctx), cell, cell_start, perm,
                               (dvec4*)pos_sorted, st);
}

extern "C" int dcm_box_counts(dcm_ctx* ctx, int64_t n, const void* pos, int32_t* box_count, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  int r = check_n(ctx, n);
  if (r) return r;
  REQUIRE(box_count && (n == 0 || pos), "dcm_box_counts: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->precision == DCM_PREC_MIXED)
    return histogram<float>(ctx, n, (const float4*)pos, box_grid<float>(ctx), box_count, st);
  return histogram<double>(ctx, n, (const dvec4*)pos, box_grid<double>(ctx), box_count, st);
}

extern "C" int dcm_detect_interface(dcm_ctx* ctx, const int32_t* box_count, uint8_t* s, uint8_t* iface,
                                    int32_t* threshold, int32_t* g, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  REQUIRE(box_count && s && iface && threshold, "dcm_detect_interface: null argument");
  return detect_interface(ctx, box_count, s, iface, threshold, g, (cudaStream_t)stream);
}

extern "C" int dcm_remove_small_components(dcm_ctx* ctx, const uint8_t* s_in, uint8_t* s_out, uint8_t* iface,
                                           dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  REQUIRE(s_in && s_out && iface && s_in != s_out, "dcm_remove_small_components: null or aliased argument");
  return remove_small_components(ctx, s_in, s_out, iface, (cudaStream_t)stream);
}

extern "C" int dcm_distance(dcm_ctx* ctx, const uint8_t* s, const uint8_t* iface, void* D, int32_t* iters,
                            dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  REQUIRE(s && iface && D, "dcm_distance: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->precision == DCM_PREC_MIXED) return distance_sweeps<float>(ctx, s, iface, (float*)D, iters, true, st);
  return distance_sweeps<double>(ctx, s, iface, (double*)D, iters, true, st);
}

extern "C" int dcm_cutoffs(dcm_ctx* ctx, int64_t n, const void* pos, const void* D, void* rc, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  int r = check_n(ctx, n);
  if (r) return r;
  REQUIRE(D && (n == 0 || (pos && rc)), "dcm_cutoffs: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->precision == DCM_PREC_MIXED)
    return assign_cutoffs<float>(ctx, n, (const float4*)pos, (const float*)D, (float*)rc, st);
  return assign_cutoffs<double>(ctx, n, (const dvec4*)pos, (const double*)D, (double*)rc, st);
}

extern "C" int dcm_forces(dcm_ctx* ctx, int64_t n, const void* pos_sorted, const void* rc, const int32_t* cell_start,
                          void* force, double* totals, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  int r = check_n(ctx, n);
  if (r) return r;
  REQUIRE(cell_start && (n == 0 || (pos_sorted && rc && force)), "dcm_forces: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->precision == DCM_PREC_MIXED)
    return lj_forces<float>(ctx, n, (const float4*)pos_sorted, (const float*)rc, cell_start, (float4*)force, totals,
                            st);
  return lj_forces<double>(ctx, n, (const dvec4*)pos_sorted, (const double*)rc, cell_start, (dvec4*)force, totals,
                           st);
}

static int check_state(dcm_ctx* ctx, const dcm_state* st, int64_t n) {
  if (!st) return set_error(ctx, DCM_ERR_INVALID_ARG, "state is NULL");
  if (st->cur != 0 && st->cur != 1) return set_error(ctx, DCM_ERR_INVALID_ARG, "state.cur must be 0 or 1");
  if (n > 0)
    for (int b = 0; b < 2; ++b)
      if (!st->pos[b] || !st->vel[b] || !st->rc[b])
        return set_error(ctx, DCM_ERR_INVALID_ARG, "state buffers pos/vel/rc must be set");
  if (n > 0 && !st->force) return set_error(ctx, DCM_ERR_INVALID_ARG, "state.force must be set");
  if ((st->id[0] == nullptr) != (st->id[1] == nullptr))
    return set_error(ctx, DCM_ERR_INVALID_ARG, "state.id needs both buffers or none");
  return DCM_OK;
}

extern "C" int dcm_step_init(dcm_ctx* ctx, dcm_state* st, int64_t n, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  int r = check_n(ctx, n);
  if (r) return r;
  if ((r = check_state(ctx, st, n))) return r;
  if (ctx->precision == DCM_PREC_MIXED) return step_init<float>(ctx, st, n, (cudaStream_t)stream);
  return step_init<double>(ctx, st, n, (cudaStream_t)stream);
}

extern "C" int dcm_step(dcm_ctx* ctx, dcm_state* st, int64_t n, double dt, int32_t nsteps, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  int r = check_n(ctx, n);
  if (r) return r;
  if ((r = check_state(ctx, st, n))) return r;
  if (nsteps < 0 || !(dt > 0.0)) return set_error(ctx, DCM_ERR_INVALID_ARG, "need nsteps >= 0 and dt > 0");
  if (ctx->precision == DCM_PREC_MIXED) return step_run<float>(ctx, st, n, dt, nsteps, (cudaStream_t)stream);
  return step_run<double>(ctx, st, n, dt, nsteps, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------
extern "C" int dcm_set_timing(dcm_ctx* ctx, int32_t capacity) {
  if (!ctx || capacity < 0 || capacity > 100000) return DCM_ERR_INVALID_ARG;
  if (capacity > ctx->ev_cap) {
    DCM_CUDA_TRY(ctx, cudaDeviceSynchronize());
    if (ctx->ev) {
      for (int64_t k = 0; k < (int64_t)DCM_NSTAGES * ctx->ev_cap * 2; ++k)
        if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
      free(ctx->ev);
    }
    int64_t total = (int64_t)DCM_NSTAGES * capacity * 2;
    ctx->ev = (cudaEvent_t*)calloc((size_t)total, sizeof(cudaEvent_t));
    ctx->ev_cap = 0;
    if (!ctx->ev) return set_error(ctx, DCM_ERR_NOMEM, "event table");
    for (int64_t k = 0; k < total; ++k) DCM_CUDA_TRY(ctx, cudaEventCreate(&ctx->ev[k]));
    ctx->ev_cap = capacity;
  }
  for (int s = 0; s < DCM_NSTAGES; ++s) ctx->ev_n[s] = 0;
  ctx->timing = capacity > 0 ? 1 : 0;
  return DCM_OK;
}

extern "C" int dcm_stage_times(dcm_ctx* ctx, double* ms, int64_t* count) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  int code = DCM_OK;
  if (ctx->ev) DCM_CUDA_TRY(ctx, cudaDeviceSynchronize());
  for (int s = 0; s < DCM_NSTAGES; ++s) {
    double t = 0.0;
    int k = ctx->ev_n[s];
    if (k > ctx->ev_cap) code = set_error(ctx, DCM_ERR_CAPACITY, "%d timed launches of stage %d exceed %d", k, s,
                                          ctx->ev_cap);
    for (int j = 0; j < k && j < ctx->ev_cap; ++j) {
      float e = 0.f;
      DCM_CUDA_TRY(ctx, cudaEventElapsedTime(&e, event_at(ctx, s, j, 0), event_at(ctx, s, j, 1)));
      t += e;
    }
    if (ms) ms[s] = t;
    if (count) count[s] = k;
    ctx->ev_n[s] = 0;
  }
  return code;
}

extern "C" int dcm_launch_count(dcm_ctx* ctx, int64_t* count, int32_t reset) {
  if (!ctx || !count) return DCM_ERR_INVALID_ARG;
  *count = ctx->launches;
  if (reset) ctx->launches = 0;
  return DCM_OK;
}

extern "C" int dcm_force_kernel(const dcm_ctx* ctx, int32_t* kernel) {
  if (!ctx || !kernel) return DCM_ERR_INVALID_ARG;
  *kernel = resolve_force_kernel(ctx);
  return DCM_OK;
}

extern "C" int dcm_accumulation(const dcm_ctx* ctx, int32_t* form) {
  if (!ctx || !form) return DCM_ERR_INVALID_ARG;
  *form = resolve_accumulation(ctx);
  return DCM_OK;
}

// ---------------------------------------------------------------------------
// differentiation
// ---------------------------------------------------------------------------
extern "C" int dcm_set_lj(dcm_ctx* ctx, int32_t ntypes, const double* eps, const double* sigma) {
  if (!ctx || !eps || !sigma) return DCM_ERR_INVALID_ARG;
  dcm_params q = ctx->p;
  q.ntypes = ntypes;
  for (int k = 0; k < 4; ++k) {
    q.eps[k] = k < ntypes ? eps[k] : 1.0;
    q.sigma[k] = k < ntypes ? sigma[k] : 1.0;
  }
  char msg[256];
  int r = dcm_validate_params(&q, msg, sizeof(msg));
  if (r) return set_error(ctx, r, "%s", msg);
  ctx->p.ntypes = ntypes;
  for (int k = 0; k < 4; ++k) {
    ctx->p.eps[k] = q.eps[k];
    ctx->p.sigma[k] = q.sigma[k];
  }
  return DCM_OK;
}

extern "C" int dcm_forces_backward(dcm_ctx* ctx, int64_t n, const void* pos_sorted, const void* rc,
                                   const int32_t* cell_start, const void* dL_dF, double dL_dE, void* dL_dpos,
                                   double* dL_dparams, dcm_stream_t stream) {
  if (!ctx) return DCM_ERR_INVALID_ARG;
  int r = check_n(ctx, n);
  if (r) return r;
  REQUIRE(cell_start && (n == 0 || (pos_sorted && rc && dL_dF && dL_dpos)), "dcm_forces_backward: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->precision == DCM_PREC_MIXED)
    return lj_adjoint<float>(ctx, n, (const float4*)pos_sorted, (const float*)rc, cell_start, (const float4*)dL_dF,
                             dL_dE, (float4*)dL_dpos, dL_dparams, st);
  return lj_adjoint<double>(ctx, n, (const dvec4*)pos_sorted, (const double*)rc, cell_start, (const dvec4*)dL_dF,
                            dL_dE, (dvec4*)dL_dpos, dL_dparams, st);
}
