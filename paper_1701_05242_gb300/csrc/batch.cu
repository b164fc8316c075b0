// Batched form: R independent systems (replicas) of different sizes stepped
// together, each stage one launch over the concatenation of all replicas.
//
// Layout: the replicas' particles are concatenated (replica r owns sorted
// slots [p0_r, p1_r)), their force cells are concatenated (replica r's cells
// start at c0_r) and so are their density boxes (b0_r).  A particle never
// leaves its replica, so its replica index is fixed (rep_of_particle); a box's
// replica index is fixed too (rep_of_box).  Because cells are concatenated in
// replica order, one exclusive scan over all cell counts gives every
// replica's cell starts as global slot indices, and the single-system scan,
// scatter and per-cell sort work unchanged on the concatenation.  The kernels
// that depend on the box geometry read it from a per-replica table.
//
// The whole K-step recomputation period can be captured once in a CUDA graph
// and replayed (dcm_batch_capture / dcm_batch_replay): every size is fixed,
// the distance sweeps run a fixed budget with device-side early exit, and no
// call inside a step waits on the host.
#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstring>
#include <new>
#include <vector>

#include "forces_core.cuh"

namespace dcm {

struct RepGeom {
  int64_t p0, p1;  // particle slots
  int64_t c0;      // first force cell
  int64_t b0;      // first density box
  int nc[3];       // force cells per dimension
  int nb[3];       // density boxes per dimension
  double L[3];     // box lengths
};

constexpr int kBatchHistBins = 4096;  // per-replica histogram of box sums
constexpr int64_t kThermoChunk = 4096;  // particles per block of the per-replica sums

}  // namespace dcm

struct dcm_batch {
  dcm_params p;
  int R;
  int precision;
  int64_t ntot, ncell_tot, nbox_tot;
  dcm_ctx base;  // scratch sized for the concatenation (shared launchers use it)
  std::vector<dcm::RepGeom> geom_h;
  dcm::RepGeom* geom;
  uint16_t* rep_of_particle;
  uint16_t* rep_of_box;
  int32_t* thr;       // [R][4]: gmin, gmax, T, unused
  int32_t* hist;      // [R][kBatchHistBins]
  void* w_i;          // per-particle virial (real)
  void* ke_i;         // per-particle kinetic energy (real)
  int32_t* np_i;      // per-particle accepted pairs
  int32_t nchunk;     // thermo reduction: chunks of at most kThermoChunk particles of one replica
  int64_t* chunk;     // [nchunk][2]: first, end particle
  int32_t* chunk0;    // [R + 1]: first chunk of each replica
  double* tpart;      // [4][nchunk]: per-chunk E, W, KE, pairs
  int force_block;    // threads per block of the force kernel
  cudaGraphExec_t graph;
  int graph_steps;
  int64_t graph_launches;  // kernels per replay
  void* graph_key[8];
};

namespace dcm {

static int berr(dcm_batch* b, int code, const char* fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->base.err, sizeof(b->base.err), fmt, ap);
    va_end(ap);
  }
  return code;
}

template <typename R>
__device__ __forceinline__ R wrapL(R x, R L) {
  if (x >= L) x -= L;
  if (x < (R)0) {
    x += L;
    if (x >= L) x = (R)0;
  }
  return x;
}

template <typename R>
__device__ __forceinline__ Grid<R> rep_cells(const RepGeom& G, R l, R il, R lx, R ilx) {
  Grid<R> g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = G.nc[d];
    g.L[d] = (R)G.L[d];
  }
  g.edge = l;
  g.inv_edge = il;
  g.edge_x = lx;
  g.inv_edge_x = ilx;
  g.ncell = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];
  return g;
}

// ---- integrate + bin ---------------------------------------------------------
template <typename R>
__global__ void k_b_kick_drift_count(int64_t n, typename RT<R>::R4* __restrict__ pos, typename RT<R>::R4* __restrict__ vel,
                                     const typename RT<R>::R4* __restrict__ force, R half_dt, R dt, R l, R il,
                                     R lx, R ilx, const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep,
                                     int32_t* __restrict__ cell, int32_t* __restrict__ slot, int32_t* __restrict__ count,
                                     int drift) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RepGeom& G = geom[rep[i]];
  auto p = pos[i];
  if (drift) {
    auto v = vel[i];
    auto f = force[i];
    v.x += half_dt * f.x;
    v.y += half_dt * f.y;
    v.z += half_dt * f.z;
    p.x = wrapL<R>(p.x + dt * v.x, (R)G.L[0]);
    p.y = wrapL<R>(p.y + dt * v.y, (R)G.L[1]);
    p.z = wrapL<R>(p.z + dt * v.z, (R)G.L[2]);
    pos[i] = p;
    vel[i] = v;
  }
  int cx = cell_coord<R>(p.x, lx, ilx, G.nc[0]);
  int cy = cell_coord<R>(p.y, l, il, G.nc[1]);
  int cz = cell_coord<R>(p.z, l, il, G.nc[2]);
  int c = (int)G.c0 + cx + G.nc[0] * (cy + G.nc[1] * cz);
  cell[i] = c;
  slot[i] = atomicAdd(count + c, 1);
}

template <typename R>
__global__ void k_b_gather(int64_t n, const int32_t* __restrict__ perm, const typename RT<R>::R4* __restrict__ p0,
                           typename RT<R>::R4* __restrict__ p1, const typename RT<R>::R4* __restrict__ v0,
                           typename RT<R>::R4* __restrict__ v1, const R* __restrict__ r0, R* __restrict__ r1,
                           const int32_t* __restrict__ id0, int32_t* __restrict__ id1) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int src = perm[k];
  p1[k] = p0[src];
  v1[k] = v0[src];
  r1[k] = r0[src];
  if (id0) id1[k] = id0[src];
}

template <typename R>
__global__ void k_b_box_count(int64_t n, const typename RT<R>::R4* __restrict__ pos, R h, R ih,
                              const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep,
                              int32_t* __restrict__ count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RepGeom& G = geom[rep[i]];
  auto p = pos[i];
  int cx = cell_coord<R>(p.x, h, ih, G.nb[0]);
  int cy = cell_coord<R>(p.y, h, ih, G.nb[1]);
  int cz = cell_coord<R>(p.z, h, ih, G.nb[2]);
  atomicAdd(count + G.b0 + cx + G.nb[0] * (cy + G.nb[1] * cz), 1);
}

// ---- interface detection (per replica) -----------------------------------------
template <int AXIS>
__global__ void k_b_box_sum(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t nbox,
                            const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep, int w) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  const RepGeom& G = geom[rep[b]];
  int64_t lb = b - G.b0;
  int nx = G.nb[0], ny = G.nb[1], nz = G.nb[2];
  int x = (int)(lb % nx), y = (int)((lb / nx) % ny), z = (int)(lb / ((int64_t)nx * ny));
  int n = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
  int c = AXIS == 0 ? x : (AXIS == 1 ? y : z);
  int64_t stride = AXIS == 0 ? 1 : (AXIS == 1 ? nx : (int64_t)nx * ny);
  int64_t base = b - (int64_t)c * stride;
  int s = 0;
  for (int a = -w; a <= w; ++a) {
    int k = (c + a) % n;
    if (k < 0) k += n;
    s += in[base + (int64_t)k * stride];
  }
  out[b] = s;
}

__global__ void k_b_thr_init(int32_t* thr, int R, int fixed) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  thr[4 * r + 0] = INT_MAX;
  thr[4 * r + 1] = INT_MIN;
  thr[4 * r + 2] = fixed;
}

__global__ void k_b_minmax(const int32_t* __restrict__ g, int64_t nbox, const uint16_t* __restrict__ rep, int32_t* thr) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int r = b < nbox ? rep[b] : -1;
  int v = b < nbox ? g[b] : 0;
  int r0 = __shfl_sync(0xffffffffu, r, 0);
  bool uniform = __all_sync(0xffffffffu, r == r0);
  if (uniform) {
    if (r0 < 0) return;
    int lo = v, hi = v;
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(thr + 4 * r0, lo);
      atomicMax(thr + 4 * r0 + 1, hi);
    }
  } else if (r >= 0) {
    atomicMin(thr + 4 * r, v);
    atomicMax(thr + 4 * r + 1, v);
  }
}

__global__ void k_b_value_hist(const int32_t* __restrict__ g, int64_t nbox, const uint16_t* __restrict__ rep,
                               const int32_t* thr, int32_t* hist, int32_t* status) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  int r = rep[b];
  int gmin = thr[4 * r], gmax = thr[4 * r + 1];
  if ((int64_t)gmax - gmin >= kBatchHistBins) {
    raise_status(status, DCM_ERR_CAPACITY);
    return;
  }
  atomicAdd(hist + (int64_t)r * kBatchHistBins + (g[b] - gmin), 1);
}

__device__ long long bsum_ll(long long v, long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  long long t = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  return t;
}

// one block per replica: integer 2-means on the replica's histogram (same
// iteration as the single-system detection)
__global__ void k_b_two_means(const int32_t* __restrict__ hist, int32_t* thr, int max_iter) {
  __shared__ long long sh[32];
  __shared__ int T_sh;
  int r = blockIdx.x;
  if (thr[4 * r + 2] >= 0) return;  // fixed threshold
  int gmin = thr[4 * r], gmax = thr[4 * r + 1];
  if ((int64_t)gmax - gmin >= kBatchHistBins) return;
  const int32_t* h = hist + (int64_t)r * kBatchHistBins;
  int Rn = gmax - gmin + 1;
  if (threadIdx.x == 0) T_sh = (int)(((long long)gmin + gmax) / 2);
  __syncthreads();
  for (int it = 0; it < max_iter; ++it) {
    int T = T_sh;
    long long n0 = 0, n1 = 0, s0 = 0, s1 = 0;
    for (int k = threadIdx.x; k < Rn; k += blockDim.x) {
      long long c = h[k], v = (long long)(gmin + k);
      if (gmin + k < T) {
        n0 += c;
        s0 += c * v;
      } else {
        n1 += c;
        s1 += c * v;
      }
    }
    n0 = bsum_ll(n0, sh);
    n1 = bsum_ll(n1, sh);
    s0 = bsum_ll(s0, sh);
    s1 = bsum_ll(s1, sh);
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
  if (threadIdx.x == 0) thr[4 * r + 2] = T_sh;
}

__global__ void k_b_segment(const int32_t* __restrict__ g, int64_t nbox, const RepGeom* __restrict__ geom,
                            const uint16_t* __restrict__ rep, const int32_t* thr, uint8_t* __restrict__ s,
                            uint8_t* __restrict__ iface) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  int r = rep[b];
  const RepGeom& G = geom[r];
  int T = thr[4 * r + 2];
  int64_t lb = b - G.b0;
  int nx = G.nb[0], ny = G.nb[1], nz = G.nb[2];
  int x = (int)(lb % nx), y = (int)((lb / nx) % ny), z = (int)(lb / ((int64_t)nx * ny));
  int me = g[b] >= T;
  int f = 0;
  if (me) {
    const int32_t* gb = g + G.b0;
    int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    int64_t row = (int64_t)nx * (y + (int64_t)ny * z);
    f |= gb[row + xm] < T;
    f |= gb[row + xp] < T;
    f |= gb[x + nx * (ym + (int64_t)ny * z)] < T;
    f |= gb[x + nx * (yp + (int64_t)ny * z)] < T;
    f |= gb[x + nx * (y + (int64_t)ny * zm)] < T;
    f |= gb[x + nx * (y + (int64_t)ny * zp)] < T;
  }
  s[b] = (uint8_t)me;
  iface[b] = (uint8_t)f;
}

// ---- distances (per replica grids, one convergence flag for all) ----------------
template <typename R>
__global__ void k_b_dist_init(const uint8_t* __restrict__ s, const uint8_t* __restrict__ iface, int64_t nbox,
                              R* __restrict__ D0, R* __restrict__ D1) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  R v = (!s[b] || iface[b]) ? (R)0 : RT<R>::inf();
  D0[b] = v;
  D1[b] = v;
}

template <typename R>
__device__ __forceinline__ R b_godunov3(R a0, R a1, R a2, R h) {
  R t;
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
  if (a0 > a1) { t = a0; a0 = a1; a1 = t; }
  R d = a0 + h;
  if (d > a1) {
    R df = a0 - a1;
    d = (R)0.5 * (a0 + a1 + sqrt((R)2 * h * h - df * df));
    if (d > a2) {
      R sa = a0 + a1 + a2;
      R sq = a0 * a0 + a1 * a1 + a2 * a2;
      R disc = sa * sa - (R)3 * (sq - h * h);
      d = (sa + sqrt(disc > (R)0 ? disc : (R)0)) / (R)3;
    }
  }
  return d;
}

template <typename R>
__global__ void k_b_dist_sweep(const R* __restrict__ Din, R* __restrict__ Dout, int64_t nbox,
                               const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep, R h, R r_grid,
                               int32_t* __restrict__ flags, int it) {
  if (it > 0 && flags[it - 1] == 0) return;
  bool changed = false;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += (int64_t)gridDim.x * blockDim.x) {
    R cur = Din[b];
    if (cur == (R)0) continue;
    const RepGeom& G = geom[rep[b]];
    int64_t lb = b - G.b0;
    int nx = G.nb[0], ny = G.nb[1], nz = G.nb[2];
    int x = (int)(lb % nx), y = (int)((lb / nx) % ny), z = (int)(lb / ((int64_t)nx * ny));
    const R* D = Din + G.b0;
    int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    int64_t row = (int64_t)nx * (y + (int64_t)ny * z);
    R a0 = fmin(D[row + xm], D[row + xp]);
    R a1 = fmin(D[x + nx * (ym + (int64_t)ny * z)], D[x + nx * (yp + (int64_t)ny * z)]);
    R a2 = fmin(D[x + nx * (y + (int64_t)ny * zm)], D[x + nx * (y + (int64_t)ny * zp)]);
    R d = b_godunov3<R>(a0, a1, a2, h);
    R out = cur;
    if (d < cur && d <= r_grid) {
      out = d;
      changed = true;
    }
    Dout[b] = out;
  }
  if (__any_sync(0xffffffffu, changed) && (threadIdx.x & 31) == 0) flags[it] = 1;
}

__global__ void k_b_dist_finish(const int32_t* flags, int sweeps, int32_t* status) {
  int first = -1;
  for (int k = 0; k < sweeps; ++k)
    if (flags[k] == 0) {
      first = k;
      break;
    }
  if (first < 0) raise_status(status, DCM_ERR_NOT_CONVERGED);
}

// ---- cutoffs ----------------------------------------------------------------------
template <typename R>
__global__ void k_b_cutoffs(int64_t n, const typename RT<R>::R4* __restrict__ pos, const R* __restrict__ D,
                            const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep, R h, R r_grid,
                            R rc_min, R rc_max, R ramp, R* __restrict__ rc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RepGeom& G = geom[rep[i]];
  auto p = ldg4(pos + i);
  int k[3];
  R t[3];
  R x[3] = {p.x, p.y, p.z};
  for (int d = 0; d < 3; ++d) {
    R q = floor(x[d] / h - (R)0.5);
    int kk = (int)q;
    if (((R)kk + (R)0.5) * h > x[d])
      --kk;
    else if (((R)kk + (R)1.5) * h <= x[d])
      ++kk;
    k[d] = kk;
    t[d] = (x[d] - ((R)kk + (R)0.5) * h) / h;
  }
  auto wrapk = [](int kk, int nn) { kk %= nn; return kk < 0 ? kk + nn : kk; };
  int nx = G.nb[0], ny = G.nb[1], nz = G.nb[2];
  int x0 = wrapk(k[0], nx), x1 = wrapk(k[0] + 1, nx);
  int y0 = wrapk(k[1], ny), y1 = wrapk(k[1] + 1, ny);
  int z0 = wrapk(k[2], nz), z1 = wrapk(k[2] + 1, nz);
  const R* Dr = D + G.b0;
  auto at = [&](int a, int b, int c) {
    R v = Dr[a + (int64_t)nx * (b + (int64_t)ny * c)];
    return v < r_grid ? v : r_grid;
  };
  auto lerp = [](R a, R b, R tt) { return fma(tt, b - a, a); };
  R c00 = lerp(at(x0, y0, z0), at(x1, y0, z0), t[0]);
  R c10 = lerp(at(x0, y1, z0), at(x1, y1, z0), t[0]);
  R c01 = lerp(at(x0, y0, z1), at(x1, y0, z1), t[0]);
  R c11 = lerp(at(x0, y1, z1), at(x1, y1, z1), t[0]);
  R delta = lerp(lerp(c00, c10, t[1]), lerp(c01, c11, t[1]), t[2]);
  R r;
  if (ramp > (R)0) {
    r = rc_max - (rc_max - rc_min) * delta / ramp;
    r = r < rc_min ? rc_min : (r > rc_max ? rc_max : r);
  } else {
    r = delta > (R)0 ? rc_min : rc_max;
  }
  rc[i] = r;
}

// ---- forces -----------------------------------------------------------------------
template <typename R, bool TYPED, bool X2, Accum M>
__global__ void k_b_forces(int64_t n, const typename RT<R>::R4* __restrict__ pos, const R* __restrict__ rc,
                           const int32_t* __restrict__ start, ForceArgs<R> a, const RepGeom* __restrict__ geom,
                           const uint16_t* __restrict__ rep, typename RT<R>::R4* __restrict__ force,
                           R* __restrict__ w_i, int32_t* __restrict__ np_i) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const RepGeom& G = geom[rep[i]];
  Grid<R> g = rep_cells<R>(G, a.g.edge, a.g.inv_edge, a.g.edge_x, a.g.inv_edge_x);
  double e = 0, w = 0;
  int np = 0;
  force[i] = force_one<R, TYPED, X2, M>(pos, start + G.c0, g, a, (int)i, ldg4(pos + i), rc[i], e, w, np);
  w_i[i] = (R)w;
  np_i[i] = np;
}

// ---- kick + per-replica thermo ----------------------------------------------------
template <typename R>
__global__ void k_b_kick(int64_t n, typename RT<R>::R4* __restrict__ vel, const typename RT<R>::R4* __restrict__ force,
                         R half_dt, R* __restrict__ ke_i) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  auto v = vel[i];
  if (force) {
    auto f = force[i];
    v.x += half_dt * f.x;
    v.y += half_dt * f.y;
    v.z += half_dt * f.z;
    vel[i] = v;
  }
  ke_i[i] = (R)0.5 * (v.x * v.x + v.y * v.y + v.z * v.z);
}

// Per-replica thermo in two fixed-order levels: one block per chunk of at
// most kThermoChunk particles of one replica (FP64 sums), then one warp per
// replica over its chunks.  thermo[4 r + {0,1,2,3}] = {E, W, KE, pairs}.
template <typename R>
__global__ void k_b_thermo_chunks(const int64_t* __restrict__ chunk, int32_t nchunk,
                                  const typename RT<R>::R4* __restrict__ force, const R* __restrict__ w_i,
                                  const R* __restrict__ ke_i, const int32_t* __restrict__ np_i,
                                  double* __restrict__ tpart) {
  __shared__ double sh[4][8];
  const int64_t p0 = chunk[2 * blockIdx.x], p1 = chunk[2 * blockIdx.x + 1];
  double v[4] = {0, 0, 0, 0};
  for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
    v[0] += (double)force[i].w;
    v[1] += (double)w_i[i];
    v[2] += (double)ke_i[i];
    v[3] += (double)np_i[i];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 4; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane == 0)
    for (int q = 0; q < 4; ++q) sh[q][wid] = v[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[threadIdx.x][k];
    tpart[(int64_t)threadIdx.x * nchunk + blockIdx.x] = t;
  }
}

__global__ void k_b_thermo_sum(const int32_t* __restrict__ chunk0, int R, int32_t nchunk,
                               const double* __restrict__ tpart, double* __restrict__ thermo) {
  const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (r >= R) return;
  const int c0 = chunk0[r], c1 = chunk0[r + 1];
  for (int q = 0; q < 4; ++q) {
    double t = 0;
    for (int c = c0 + lane; c < c1; c += 32) t += tpart[(int64_t)q * nchunk + c];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) thermo[4 * r + q] = t;
  }
}

// ---- orchestration ------------------------------------------------------------------
template <typename R>
static int b_recompute(dcm_batch* b, const typename RT<R>::R4* pos, R* rc, cudaStream_t st) {
  dcm_ctx* ctx = &b->base;
  const dcm_params& p = b->p;
  int64_t n = b->ntot, nb = b->nbox_tot;
  unsigned gp = (unsigned)((n + 255) / 256), gb = (unsigned)((nb + 255) / 256);
  const int32_t* counts = ctx->cell_count;
  if (p.h != p.l || p.lx != p.l) {
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->box_count, 0, sizeof(int32_t) * nb, st));
    if (n > 0)
      DCM_LAUNCH(ctx, k_b_box_count<R>, gp, 256, 0, st, n, pos, (R)p.h, (R)(1.0 / p.h), b->geom, b->rep_of_particle,
                 ctx->box_count);
    counts = ctx->box_count;
  }
  stage_begin(ctx, DCM_STAGE_DETECT, st);
  int w = p.smooth_w;
  DCM_LAUNCH(ctx, k_b_box_sum<0>, gb, 256, 0, st, counts, ctx->g, nb, b->geom, b->rep_of_box, w);
  DCM_LAUNCH(ctx, k_b_box_sum<1>, gb, 256, 0, st, ctx->g, ctx->g_tmp, nb, b->geom, b->rep_of_box, w);
  DCM_LAUNCH(ctx, k_b_box_sum<2>, gb, 256, 0, st, ctx->g_tmp, ctx->g, nb, b->geom, b->rep_of_box, w);
  DCM_LAUNCH(ctx, k_b_thr_init, (unsigned)((b->R + 63) / 64), 64, 0, st, b->thr, b->R, p.threshold);
  if (p.threshold < 0) {
    DCM_LAUNCH(ctx, k_b_minmax, gb, 256, 0, st, ctx->g, nb, b->rep_of_box, b->thr);
    DCM_CUDA_TRY(ctx, cudaMemsetAsync(b->hist, 0, sizeof(int32_t) * (size_t)b->R * kBatchHistBins, st));
    DCM_LAUNCH(ctx, k_b_value_hist, gb, 256, 0, st, ctx->g, nb, b->rep_of_box, b->thr, b->hist, ctx->status);
    DCM_LAUNCH(ctx, k_b_two_means, (unsigned)b->R, 1024, 0, st, b->hist, b->thr, 64);
  }
  DCM_LAUNCH(ctx, k_b_segment, gb, 256, 0, st, ctx->g, nb, b->geom, b->rep_of_box, b->thr, ctx->s, ctx->iface);
  stage_end(ctx, DCM_STAGE_DETECT, st);
  stage_begin(ctx, DCM_STAGE_DISTANCE, st);
  R* D0 = (R*)ctx->D[0];
  R* D1 = (R*)ctx->D[1];
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->flags, 0, sizeof(int32_t) * (size_t)(p.iter_max + 2), st));
  DCM_LAUNCH(ctx, k_b_dist_init<R>, gb, 256, 0, st, ctx->s, ctx->iface, nb, D0, D1);
  int budget = (int)std::ceil(8.0 * p.r_grid / p.h) + 8;
  budget = std::min(budget + (budget & 1), p.iter_max + (p.iter_max & 1));
  unsigned gs = (unsigned)std::min<int64_t>((nb + 255) / 256, 152 * 8);
  R* buf[2] = {D0, D1};
  for (int it = 0; it < budget; ++it)
    DCM_LAUNCH(ctx, k_b_dist_sweep<R>, gs, 256, 0, st, buf[it & 1], buf[(it + 1) & 1], nb, b->geom, b->rep_of_box,
               (R)p.h, (R)p.r_grid, ctx->flags, it);
  DCM_LAUNCH(ctx, k_b_dist_finish, 1, 1, 0, st, ctx->flags, budget, ctx->status);
  stage_end(ctx, DCM_STAGE_DISTANCE, st);
  stage_begin(ctx, DCM_STAGE_CUTOFFS, st);
  if (n > 0)
    DCM_LAUNCH(ctx, k_b_cutoffs<R>, gp, 256, 0, st, n, pos, D0, b->geom, b->rep_of_particle, (R)p.h, (R)p.r_grid,
               (R)p.rc_min, (R)p.rc_max, (R)p.ramp, rc);
  stage_end(ctx, DCM_STAGE_CUTOFFS, st);
  return check_launch(ctx, "batch recompute");
}

// The batched force kernel for the LJ table and the accumulation form
// (DCM_ACC_*, resolved as for a single system).
template <typename R>
static auto b_force_kernel(bool typed, int ntypes, int acc) {
  using K = void (*)(int64_t, const typename RT<R>::R4*, const R*, const int32_t*, ForceArgs<R>, const RepGeom*,
                     const uint16_t*, typename RT<R>::R4*, R*, int32_t*);
  if constexpr (sizeof(R) == 8) {
    return typed ? (K)k_b_forces<R, true, false, Accum::kPlain> : (K)k_b_forces<R, false, false, Accum::kPlain>;
  } else {
    if (typed && ntypes > 2)
      return acc == DCM_ACC_FP32 ? (K)k_b_forces<R, true, false, Accum::kPlain>
                                 : (acc == DCM_ACC_ROW_FP64 || acc == DCM_ACC_PAIR_FP64)
                                       ? (K)k_b_forces<R, true, false, Accum::kRowF64>
                                       : (K)k_b_forces<R, true, false, Accum::kRowKahan>;
    switch (acc) {
      case DCM_ACC_FP32: return typed ? (K)k_b_forces<R, true, true, Accum::kPlain> : (K)k_b_forces<R, false, true, Accum::kPlain>;
      case DCM_ACC_ROW_FP64: return typed ? (K)k_b_forces<R, true, true, Accum::kRowF64> : (K)k_b_forces<R, false, true, Accum::kRowF64>;
      case DCM_ACC_PAIR_KAHAN: return typed ? (K)k_b_forces<R, true, true, Accum::kPairKahan> : (K)k_b_forces<R, false, true, Accum::kPairKahan>;
      case DCM_ACC_PAIR_FP64: return typed ? (K)k_b_forces<R, true, true, Accum::kPairF64> : (K)k_b_forces<R, false, true, Accum::kPairF64>;
      default: return typed ? (K)k_b_forces<R, true, true, Accum::kRowKahan> : (K)k_b_forces<R, false, true, Accum::kRowKahan>;
    }
  }
}

template <typename R>
static int b_forces_thermo(dcm_batch* b, const typename RT<R>::R4* pos, const R* rc, typename RT<R>::R4* force,
                           typename RT<R>::R4* vel, R half_dt, bool kick, double* thermo, cudaStream_t st) {
  dcm_ctx* ctx = &b->base;
  int64_t n = b->ntot;
  if (n > 0) {
    ForceArgs<R> a;
    a.g.edge = (R)b->p.l;
    a.g.inv_edge = (R)(1.0 / b->p.l);
    a.g.edge_x = (R)b->p.lx;
    a.g.inv_edge_x = (R)(1.0 / b->p.lx);
    LJTable t = lj_table(b->p);
    a.ntypes = t.ntypes;
    for (int k = 0; k < 16; ++k) {
      a.eps24[k] = (R)t.deps24[k];
      a.eps4[k] = (R)t.deps4[k];
      a.sig2[k] = (R)t.dsig2[k];
    }
    a.shift = b->p.shift_energy;
    a.rc_max = (R)b->p.rc_max;
    int bs = b->force_block;
    // the packed loop in FP32 for one type, and for one or two types with
    // their own eps and sigma; the scalar loop otherwise
    auto kern = b_force_kernel<R>(lj_general(t), t.ntypes, resolve_accumulation(ctx));
    stage_begin(ctx, DCM_STAGE_FORCES, st);
    DCM_LAUNCH(ctx, kern, (unsigned)((n + bs - 1) / bs), bs, 0, st, n, pos, rc, ctx->cell_start, a, b->geom,
               b->rep_of_particle, force, (R*)b->w_i, b->np_i);
    stage_end(ctx, DCM_STAGE_FORCES, st);
    stage_begin(ctx, DCM_STAGE_KICK, st);
    DCM_LAUNCH(ctx, k_b_kick<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, vel, kick ? force : nullptr, half_dt,
               (R*)b->ke_i);
    if (b->nchunk > 0)
      DCM_LAUNCH(ctx, k_b_thermo_chunks<R>, (unsigned)b->nchunk, 256, 0, st, b->chunk, b->nchunk, force,
                 (const R*)b->w_i, (const R*)b->ke_i, b->np_i, b->tpart);
    DCM_LAUNCH(ctx, k_b_thermo_sum, (unsigned)((b->R + 7) / 8), 256, 0, st, b->chunk0, b->R, b->nchunk, b->tpart,
               thermo);
    stage_end(ctx, DCM_STAGE_KICK, st);
  }
  return check_launch(ctx, "batch forces");
}

template <typename R>
static int b_bin_gather(dcm_batch* b, dcm_state* s, bool drift, R hdt, R dt, cudaStream_t st) {
  using R4 = typename RT<R>::R4;
  dcm_ctx* ctx = &b->base;
  int64_t n = b->ntot;
  int c = s->cur, o = 1 - c;
  stage_begin(ctx, DCM_STAGE_KICK_DRIFT, st);
  DCM_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cell_count, 0, sizeof(int32_t) * b->ncell_tot, st));
  if (n > 0)
    DCM_LAUNCH(ctx, k_b_kick_drift_count<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, (R4*)s->pos[c],
               (R4*)s->vel[c], (const R4*)s->force, hdt, dt, (R)b->p.l, (R)(1.0 / b->p.l), (R)b->p.lx,
               (R)(1.0 / b->p.lx), b->geom,
               b->rep_of_particle, ctx->cell, ctx->slot, ctx->cell_count, drift ? 1 : 0);
  stage_end(ctx, DCM_STAGE_KICK_DRIFT, st);
  stage_begin(ctx, DCM_STAGE_BIN, st);
  int r = exclusive_scan(ctx, ctx->cell_count, ctx->cell_start, b->ncell_tot, st);
  if (r) return r;
  if ((r = scatter_sort(ctx, n, ctx->cell, ctx->slot, ctx->cell_start, b->ncell_tot, ctx->perm, st))) return r;
  bool ids = s->id[c] && s->id[o];
  if (n > 0)
    DCM_LAUNCH(ctx, k_b_gather<R>, (unsigned)((n + 255) / 256), 256, 0, st, n, ctx->perm, (const R4*)s->pos[c],
               (R4*)s->pos[o], (const R4*)s->vel[c], (R4*)s->vel[o], (const R*)s->rc[c], (R*)s->rc[o],
               ids ? s->id[c] : nullptr, ids ? s->id[o] : nullptr);
  stage_end(ctx, DCM_STAGE_BIN, st);
  return check_launch(ctx, "batch bin");
}

template <typename R>
static int b_init(dcm_batch* b, dcm_state* s, cudaStream_t st) {
  using R4 = typename RT<R>::R4;
  int r = b_bin_gather<R>(b, s, false, (R)0, (R)0, st);
  if (r) return r;
  int o = 1 - s->cur;
  if ((r = b_recompute<R>(b, (const R4*)s->pos[o], (R*)s->rc[o], st))) return r;
  if ((r = b_forces_thermo<R>(b, (const R4*)s->pos[o], (const R*)s->rc[o], (R4*)s->force, (R4*)s->vel[o], (R)0,
                              false, s->thermo, st)))
    return r;
  s->cur = o;
  s->t = 0;
  return DCM_OK;
}

template <typename R>
static int b_steps(dcm_batch* b, dcm_state* s, double dt, int nsteps, cudaStream_t st) {
  using R4 = typename RT<R>::R4;
  R hdt = (R)(0.5 * dt), rdt = (R)dt;
  int K = b->p.recompute_every;
  for (int k = 0; k < nsteps; ++k) {
    int r = b_bin_gather<R>(b, s, true, hdt, rdt, st);
    if (r) return r;
    int o = 1 - s->cur;
    s->t += 1;
    if (s->t % K == 0)
      if ((r = b_recompute<R>(b, (const R4*)s->pos[o], (R*)s->rc[o], st))) return r;
    if ((r = b_forces_thermo<R>(b, (const R4*)s->pos[o], (const R*)s->rc[o], (R4*)s->force, (R4*)s->vel[o], hdt,
                                true, s->thermo, st)))
      return r;
    s->cur = o;
  }
  return DCM_OK;
}

}  // namespace dcm

using namespace dcm;

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" void dcm_batch_destroy(dcm_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  dcm_ctx* c = &b->base;
  void* dev[] = {c->status, c->slot,  c->cell,  c->perm,   c->cell_start, c->cell_count, c->scan_part,
                 c->box_count, c->g,   c->g_tmp, c->s,      c->iface,      c->D[0],       c->D[1],
                 c->flags,  c->red,   c->red_tmp, c->totals, b->geom,       b->rep_of_particle, b->rep_of_box,
                 b->thr,    b->hist,  b->w_i,   b->ke_i,   b->np_i, b->chunk, b->chunk0, b->tpart};
  for (void* q : dev)
    if (q) cudaFree(q);
  if (c->host_status) cudaFreeHost(c->host_status);
  if (c->ev) {
    for (int64_t k = 0; k < (int64_t)DCM_NSTAGES * c->ev_cap * 2; ++k)
      if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    free(c->ev);
  }
  delete b;
}

extern "C" int dcm_batch_create(const dcm_params* p, int32_t R, const double* boxes, const int64_t* counts,
                                dcm_batch** out) {
  if (!p || !boxes || !counts || !out || R < 1 || R > 65535) return DCM_ERR_INVALID_ARG;
  *out = nullptr;
  if (p->skin != 0.0) return DCM_ERR_INVALID_ARG;  // the batched form steps over cell lists only
  if (p->min_component != 0) return DCM_ERR_INVALID_ARG;  // no bubble filter in the batched form
  std::vector<RepGeom> geom((size_t)R);
  int64_t ntot = 0, nctot = 0, nbtot = 0;
  for (int r = 0; r < R; ++r) {
    dcm_params q = *p;
    for (int d = 0; d < 3; ++d) q.box[d] = boxes[3 * r + d];
    q.n_max = counts[r];
    int v = dcm_validate_params(&q, nullptr, 0);
    if (v) return v;
    if (counts[r] < 0) return DCM_ERR_INVALID_ARG;
    int64_t nc[3], nb[3];
    dcm_grid_dims(&q, nc, nb);
    RepGeom& G = geom[(size_t)r];
    G.p0 = ntot;
    G.p1 = ntot + counts[r];
    G.c0 = nctot;
    G.b0 = nbtot;
    for (int d = 0; d < 3; ++d) {
      G.nc[d] = (int)nc[d];
      G.nb[d] = (int)nb[d];
      G.L[d] = (double)nc[d] * (d == 0 && p->lx > 0.0 ? p->lx : p->l);
    }
    ntot += counts[r];
    nctot += nc[0] * nc[1] * nc[2];
    nbtot += nb[0] * nb[1] * nb[2];
  }
  if (ntot >= 0x7fffffffLL || nctot >= 0x7fffffffLL || nbtot >= 0x7fffffffLL) return DCM_ERR_CAPACITY;
  dcm_batch* b = new (std::nothrow) dcm_batch();
  if (!b) return DCM_ERR_NOMEM;
  memset(&b->base, 0, sizeof(b->base));
  b->p = *p;
  if (!(b->p.lx > 0.0)) b->p.lx = b->p.l;
  if (!(b->p.ramp > 0.0)) b->p.ramp = b->p.rc_max - b->p.rc_min;
  if (!(b->p.r_grid > 0.0)) b->p.r_grid = b->p.ramp + 2.0 * b->p.h;
  b->R = R;
  b->precision = p->precision;
  b->ntot = ntot;
  b->ncell_tot = nctot;
  b->nbox_tot = nbtot;
  b->geom_h = geom;
  b->geom = nullptr;
  b->rep_of_particle = nullptr;
  b->rep_of_box = nullptr;
  b->thr = nullptr;
  b->hist = nullptr;
  b->w_i = b->ke_i = nullptr;
  b->np_i = nullptr;
  b->nchunk = 0;
  b->chunk = nullptr;
  b->chunk0 = nullptr;
  b->tpart = nullptr;
  b->force_block = 128;
  b->graph = nullptr;
  b->graph_steps = 0;
  b->graph_launches = 0;
  memset(b->graph_key, 0, sizeof(b->graph_key));
  dcm_ctx* c = &b->base;
  c->p = b->p;
  c->precision = p->precision;
  c->ncell = nctot;
  c->nbox = nbtot;
  c->n_max = ntot;
  cudaGetDevice(&c->device);
  int64_t rs = p->precision == DCM_PREC_FP64 ? 8 : 4;
  int64_t nm = ntot > 0 ? ntot : 1;
  int64_t big = std::max(nctot, nbtot);
  c->scan_cap = (big + kScanTile - 1) / kScanTile + 1;
  c->red_cap = ((nm + 255) / 256 + 1) * 8;
  bool ok = true;
  auto alloc = [&](void** ptr, int64_t bytes) {
    if (ok && cudaMalloc(ptr, (size_t)(bytes > 0 ? bytes : 16)) != cudaSuccess) ok = false;
  };
  alloc((void**)&c->status, 16);
  alloc((void**)&c->slot, 4 * nm);
  alloc((void**)&c->cell, 4 * nm);
  alloc((void**)&c->perm, 4 * nm);
  alloc((void**)&c->cell_start, 4 * (nctot + 1));
  alloc((void**)&c->cell_count, 4 * nctot);
  alloc((void**)&c->scan_part, 4 * c->scan_cap);
  alloc((void**)&c->box_count, 4 * nbtot);
  alloc((void**)&c->g, 4 * nbtot);
  alloc((void**)&c->g_tmp, 4 * nbtot);
  alloc((void**)&c->s, nbtot);
  alloc((void**)&c->iface, nbtot);
  alloc(&c->D[0], rs * nbtot);
  alloc(&c->D[1], rs * nbtot);
  alloc((void**)&c->flags, 4 * (int64_t)(p->iter_max + 2));
  alloc((void**)&c->red, 8 * 3 * c->red_cap);
  alloc((void**)&c->red_tmp, 8 * 8 * 256);
  alloc((void**)&c->totals, 8 * 8);
  alloc((void**)&b->geom, (int64_t)sizeof(RepGeom) * R);
  alloc((void**)&b->rep_of_particle, 2 * nm);
  alloc((void**)&b->rep_of_box, 2 * nbtot);
  alloc((void**)&b->thr, 16 * (int64_t)R);
  alloc((void**)&b->hist, 4 * (int64_t)R * kBatchHistBins);
  alloc(&b->w_i, rs * nm);
  alloc(&b->ke_i, rs * nm);
  alloc((void**)&b->np_i, 4 * nm);
  std::vector<int64_t> ch;
  std::vector<int32_t> ch0((size_t)R + 1, 0);
  for (int r = 0; r < R; ++r) {
    ch0[(size_t)r] = (int32_t)(ch.size() / 2);
    for (int64_t a = geom[(size_t)r].p0; a < geom[(size_t)r].p1; a += kThermoChunk) {
      ch.push_back(a);
      ch.push_back(std::min(a + kThermoChunk, geom[(size_t)r].p1));
    }
  }
  b->nchunk = (int32_t)(ch.size() / 2);
  ch0[(size_t)R] = b->nchunk;
  alloc((void**)&b->chunk, 8 * (int64_t)ch.size());
  alloc((void**)&b->chunk0, 4 * ((int64_t)R + 1));
  alloc((void**)&b->tpart, 8 * 4 * (int64_t)std::max<int32_t>(b->nchunk, 1));
  if (ok && cudaMallocHost((void**)&c->host_status, 16) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    dcm_batch_destroy(b);
    return DCM_ERR_NOMEM;
  }
  std::vector<uint16_t> rp((size_t)nm, 0), rb((size_t)(nbtot > 0 ? nbtot : 1), 0);
  for (int r = 0; r < R; ++r) {
    for (int64_t i = geom[r].p0; i < geom[r].p1; ++i) rp[(size_t)i] = (uint16_t)r;
    int64_t nbr = (int64_t)geom[r].nb[0] * geom[r].nb[1] * geom[r].nb[2];
    for (int64_t k = 0; k < nbr; ++k) rb[(size_t)(geom[r].b0 + k)] = (uint16_t)r;
  }
  if (cudaMemcpy(b->geom, geom.data(), sizeof(RepGeom) * R, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->rep_of_particle, rp.data(), 2 * rp.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->rep_of_box, rb.data(), 2 * (size_t)nbtot, cudaMemcpyHostToDevice) != cudaSuccess ||
      (!ch.empty() && cudaMemcpy(b->chunk, ch.data(), 8 * ch.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(b->chunk0, ch0.data(), 4 * ch0.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->status, 0, 16) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    dcm_batch_destroy(b);
    return DCM_ERR_CUDA;
  }
  *out = b;
  return DCM_OK;
}

extern "C" const char* dcm_batch_last_error(const dcm_batch* b) { return b ? b->base.err : "null batch"; }

extern "C" int dcm_batch_offsets(const dcm_batch* b, int64_t* offsets) {
  if (!b || !offsets) return DCM_ERR_INVALID_ARG;
  for (int r = 0; r < b->R; ++r) offsets[r] = b->geom_h[(size_t)r].p0;
  offsets[b->R] = b->ntot;
  return DCM_OK;
}

extern "C" int dcm_batch_set_force_block(dcm_batch* b, int32_t threads) {
  if (!b || (threads != 64 && threads != 128 && threads != 256)) return DCM_ERR_INVALID_ARG;
  b->force_block = threads;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return DCM_OK;
}

static int batch_check_state(dcm_batch* b, const dcm_state* s) {
  if (!s || (s->cur != 0 && s->cur != 1)) return berr(b, DCM_ERR_INVALID_ARG, "bad state");
  if (b->ntot > 0)
    for (int k = 0; k < 2; ++k)
      if (!s->pos[k] || !s->vel[k] || !s->rc[k]) return berr(b, DCM_ERR_INVALID_ARG, "state buffers must be set");
  if (b->ntot > 0 && (!s->force || !s->thermo)) return berr(b, DCM_ERR_INVALID_ARG, "state.force/thermo must be set");
  if ((s->id[0] == nullptr) != (s->id[1] == nullptr)) return berr(b, DCM_ERR_INVALID_ARG, "id needs both buffers");
  return DCM_OK;
}

extern "C" int dcm_batch_step_init(dcm_batch* b, dcm_state* s, dcm_stream_t stream) {
  if (!b) return DCM_ERR_INVALID_ARG;
  int r = batch_check_state(b, s);
  if (r) return r;
  if (b->precision == DCM_PREC_MIXED) return b_init<float>(b, s, (cudaStream_t)stream);
  return b_init<double>(b, s, (cudaStream_t)stream);
}

extern "C" int dcm_batch_step(dcm_batch* b, dcm_state* s, double dt, int32_t nsteps, dcm_stream_t stream) {
  if (!b) return DCM_ERR_INVALID_ARG;
  int r = batch_check_state(b, s);
  if (r) return r;
  if (nsteps < 0 || !(dt > 0.0)) return berr(b, DCM_ERR_INVALID_ARG, "need nsteps >= 0 and dt > 0");
  if (b->precision == DCM_PREC_MIXED) return b_steps<float>(b, s, dt, nsteps, (cudaStream_t)stream);
  return b_steps<double>(b, s, dt, nsteps, (cudaStream_t)stream);
}

extern "C" int dcm_batch_capture(dcm_batch* b, dcm_state* s, double dt, dcm_stream_t stream) {
  if (!b) return DCM_ERR_INVALID_ARG;
  int r = batch_check_state(b, s);
  if (r) return r;
  if (!stream) return berr(b, DCM_ERR_INVALID_ARG, "graph capture needs a non-default stream");
  int K = b->p.recompute_every;
  if (s->t % K != 0) return berr(b, DCM_ERR_INVALID_ARG, "capture must start at a recomputation step (t %% K == 0)");
  if (!(dt > 0.0)) return berr(b, DCM_ERR_INVALID_ARG, "dt must be positive");
  int steps = (K % 2 == 0) ? K : 2 * K;  // even: the double buffers return to the same side
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaStream_t st = (cudaStream_t)stream;
  dcm_state tmp = *s;
  int64_t launches0 = b->base.launches;
  int timing = b->base.timing;
  b->base.timing = 0;  // no event records inside the graph
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return berr(b, DCM_ERR_CUDA, "cudaStreamBeginCapture failed");
  r = (b->precision == DCM_PREC_MIXED) ? b_steps<float>(b, &tmp, dt, steps, st) : b_steps<double>(b, &tmp, dt, steps, st);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  b->base.timing = timing;
  if (r) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (e != cudaSuccess || !graph) return berr(b, DCM_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return berr(b, DCM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  b->graph_steps = steps;
  b->graph_launches = b->base.launches - launches0;
  b->base.launches = launches0;
  void* key[8] = {s->pos[0], s->pos[1], s->vel[0], s->vel[1], s->rc[0], s->rc[1], s->force, s->thermo};
  memcpy(b->graph_key, key, sizeof(key));
  return DCM_OK;
}

extern "C" int dcm_batch_replay(dcm_batch* b, dcm_state* s, int32_t ngraphs, dcm_stream_t stream) {
  if (!b || !s || ngraphs < 0) return DCM_ERR_INVALID_ARG;
  if (!b->graph) return berr(b, DCM_ERR_INVALID_ARG, "no captured graph");
  void* key[8] = {s->pos[0], s->pos[1], s->vel[0], s->vel[1], s->rc[0], s->rc[1], s->force, s->thermo};
  if (memcmp(key, b->graph_key, sizeof(key)) != 0)
    return berr(b, DCM_ERR_INVALID_ARG, "state buffers differ from the captured ones");
  for (int k = 0; k < ngraphs; ++k) {
    cudaError_t e = cudaGraphLaunch(b->graph, (cudaStream_t)stream);
    if (e != cudaSuccess) return berr(b, DCM_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    b->base.launches += b->graph_launches;
    s->t += b->graph_steps;
  }
  return DCM_OK;
}

extern "C" int dcm_batch_graph_steps(const dcm_batch* b) { return b ? b->graph_steps : 0; }

extern "C" int dcm_batch_status(dcm_batch* b, dcm_stream_t stream) {
  if (!b) return DCM_ERR_INVALID_ARG;
  return dcm_status(&b->base, stream);
}

extern "C" int dcm_batch_set_timing(dcm_batch* b, int32_t capacity) {
  return b ? dcm_set_timing(&b->base, capacity) : DCM_ERR_INVALID_ARG;
}

extern "C" int dcm_batch_stage_times(dcm_batch* b, double* ms, int64_t* count) {
  return b ? dcm_stage_times(&b->base, ms, count) : DCM_ERR_INVALID_ARG;
}

extern "C" int dcm_batch_launch_count(dcm_batch* b, int64_t* count, int32_t reset) {
  return b ? dcm_launch_count(&b->base, count, reset) : DCM_ERR_INVALID_ARG;
}
