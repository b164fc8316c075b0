// Batched form: shared declarations and the per-element device code of its
// stages, used both by the per-stage kernels (batch.cu) and by the persistent
// kernel (batch_persist.cu, two launches per timestep).
//
// Layout: the replicas' particles are concatenated (replica r owns sorted
// slots [p0_r, p1_r)), their force cells are concatenated (replica r's cells
// start at c0_r) and so are their density boxes (b0_r).  A particle never
// leaves its replica, so its replica index is fixed (rep_of_particle); a box's
// replica index is fixed too (rep_of_box).  Because cells are concatenated in
// replica order, one exclusive scan over all cell counts gives every
// replica's cell starts as global slot indices.
#pragma once

#include <climits>
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

constexpr int kBatchHistBins = 4096;    // per-replica histogram of box sums
constexpr int64_t kThermoChunk = 4096;  // particles per block of the per-replica sums
constexpr int kQueueTile = 32;          // default particles per work item of the persistent force phase

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
  // persistent form (two cooperative launches per timestep)
  int persistent;          // 1: dcm_batch_step runs the persistent kernel (default)
  int2* tiles;             // [ntiles]: (replica, first particle) of each work item of the force phase
  int32_t ntiles;
  int32_t tile;            // particles per work item (a multiple of 32)
  uint32_t* sync;          // [4]: barrier count, barrier generation, abort flag, force-queue head
  int32_t* scan_blk;       // [grid]: per-block totals of the persistent scan
  int32_t pgrid;           // blocks of the persistent launch (co-resident), 0 until sized
  int64_t wait_budget;     // nanoseconds a barrier wait may take before it reports DCM_ERR_TIMEOUT
  unsigned long long* pacc;  // stage timing of the persistent plan: ns and runs per stage, last stamp
};

namespace dcm {

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
// Half kick and drift of particle i (if drift), then its cell and its rank
// among the particles counted into that cell so far.
template <typename R>
__device__ __forceinline__ void b_kick_drift_count(int64_t i, typename RT<R>::R4* __restrict__ pos,
                                                   typename RT<R>::R4* __restrict__ vel,
                                                   const typename RT<R>::R4* __restrict__ force, R half_dt, R dt, R l,
                                                   R il, R lx, R ilx, const RepGeom* __restrict__ geom,
                                                   const uint16_t* __restrict__ rep, int32_t* __restrict__ cell,
                                                   int32_t* __restrict__ slot, int32_t* __restrict__ count,
                                                   int drift) {
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
__device__ __forceinline__ void b_gather(int64_t k, const int32_t* __restrict__ perm,
                                         const typename RT<R>::R4* __restrict__ p0, typename RT<R>::R4* __restrict__ p1,
                                         const typename RT<R>::R4* __restrict__ v0, typename RT<R>::R4* __restrict__ v1,
                                         const R* __restrict__ r0, R* __restrict__ r1, const int32_t* __restrict__ id0,
                                         int32_t* __restrict__ id1) {
  int src = perm[k];
  p1[k] = p0[src];
  v1[k] = v0[src];
  r1[k] = r0[src];
  if (id0) id1[k] = id0[src];
}

// Insertion sort of one cell's entries perm[b .. e) by input index (the
// binning's stable order).
__device__ __forceinline__ void b_sort_cell(int b, int e, int32_t* __restrict__ perm) {
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

template <typename R>
__device__ __forceinline__ void b_box_count(int64_t i, const typename RT<R>::R4* __restrict__ pos, R h, R ih,
                                            const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep,
                                            int32_t* __restrict__ count) {
  const RepGeom& G = geom[rep[i]];
  auto p = pos[i];
  int cx = cell_coord<R>(p.x, h, ih, G.nb[0]);
  int cy = cell_coord<R>(p.y, h, ih, G.nb[1]);
  int cz = cell_coord<R>(p.z, h, ih, G.nb[2]);
  atomicAdd(count + G.b0 + cx + G.nb[0] * (cy + G.nb[1] * cz), 1);
}

// ---- interface detection (per replica) -----------------------------------------
template <int AXIS>
__device__ __forceinline__ void b_box_sum(int64_t b, const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                          const RepGeom* __restrict__ geom, const uint16_t* __restrict__ rep, int w) {
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

__device__ __forceinline__ void b_thr_init(int r, int32_t* thr, int fixed) {
  thr[4 * r + 0] = INT_MAX;
  thr[4 * r + 1] = INT_MIN;
  thr[4 * r + 2] = fixed;
}

// Per-replica min and max of the box sums.  All 32 lanes of the warp must
// call it together (b >= nbox: no box); a warp whose boxes share one replica
// reduces before its atomics.
__device__ __forceinline__ void b_minmax(int64_t b, const int32_t* __restrict__ g, int64_t nbox,
                                         const uint16_t* __restrict__ rep, int32_t* thr) {
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

__device__ __forceinline__ void b_value_hist(int64_t b, const int32_t* __restrict__ g,
                                             const uint16_t* __restrict__ rep, const int32_t* thr, int32_t* hist,
                                             int32_t* status) {
  int r = rep[b];
  int gmin = thr[4 * r], gmax = thr[4 * r + 1];
  if ((int64_t)gmax - gmin >= kBatchHistBins) {
    raise_status(status, DCM_ERR_CAPACITY);
    return;
  }
  atomicAdd(hist + (int64_t)r * kBatchHistBins + (g[b] - gmin), 1);
}

// Block-wide sum (every thread of the block calls it; sh holds 32 slots).
__device__ __forceinline__ long long b_block_sum_ll(long long v, long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  long long t = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
  return t;
}

// Integer 2-means of replica r on its histogram, by the whole block (the
// same iteration as the single-system detection).
__device__ __forceinline__ void b_two_means(int r, const int32_t* __restrict__ hist, int32_t* thr, int max_iter) {
  __shared__ long long sh[32];
  __shared__ int T_sh;
  if (thr[4 * r + 2] >= 0) return;  // fixed threshold (uniform over the block)
  int gmin = thr[4 * r], gmax = thr[4 * r + 1];
  if ((int64_t)gmax - gmin >= kBatchHistBins) return;
  const int32_t* h = hist + (int64_t)r * kBatchHistBins;
  int Rn = gmax - gmin + 1;
  __syncthreads();
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
    n0 = b_block_sum_ll(n0, sh);
    n1 = b_block_sum_ll(n1, sh);
    s0 = b_block_sum_ll(s0, sh);
    s1 = b_block_sum_ll(s1, sh);
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
  __syncthreads();
}

__device__ __forceinline__ void b_segment(int64_t b, const int32_t* __restrict__ g, const RepGeom* __restrict__ geom,
                                          const uint16_t* __restrict__ rep, const int32_t* thr,
                                          uint8_t* __restrict__ s, uint8_t* __restrict__ iface) {
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
__device__ __forceinline__ void b_dist_init(int64_t b, const uint8_t* __restrict__ s,
                                            const uint8_t* __restrict__ iface, R* __restrict__ D0,
                                            R* __restrict__ D1) {
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

// Jacobi update of box b from Din into Dout; true if its value changed.
// COH: the iterates read through L2 (__ldcg), for kernels whose blocks read
// what other blocks wrote earlier in the same launch (behind a grid barrier).
template <typename R, bool COH>
__device__ __forceinline__ R b_dld(const R* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

template <typename R, bool COH = false>
__device__ __forceinline__ bool b_dist_update(int64_t b, const R* Din, R* Dout, const RepGeom* __restrict__ geom,
                                              const uint16_t* __restrict__ rep, R h, R r_grid) {
  R cur = b_dld<R, COH>(Din + b);
  if (cur == (R)0) return false;
  const RepGeom& G = geom[rep[b]];
  int64_t lb = b - G.b0;
  int nx = G.nb[0], ny = G.nb[1], nz = G.nb[2];
  int x = (int)(lb % nx), y = (int)((lb / nx) % ny), z = (int)(lb / ((int64_t)nx * ny));
  const R* D = Din + G.b0;
  int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
  int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
  int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
  int64_t row = (int64_t)nx * (y + (int64_t)ny * z);
  R a0 = fmin(b_dld<R, COH>(D + row + xm), b_dld<R, COH>(D + row + xp));
  R a1 = fmin(b_dld<R, COH>(D + x + nx * (ym + (int64_t)ny * z)), b_dld<R, COH>(D + x + nx * (yp + (int64_t)ny * z)));
  R a2 = fmin(b_dld<R, COH>(D + x + nx * (y + (int64_t)ny * zm)), b_dld<R, COH>(D + x + nx * (y + (int64_t)ny * zp)));
  R d = b_godunov3<R>(a0, a1, a2, h);
  R out = cur;
  bool changed = false;
  if (d < cur && d <= r_grid) {
    out = d;
    changed = true;
  }
  Dout[b] = out;
  return changed;
}

// ---- cutoffs ----------------------------------------------------------------------
template <typename R, bool NC = true>
__device__ __forceinline__ void b_cutoffs(int64_t i, const typename RT<R>::R4* __restrict__ pos,
                                          const R* __restrict__ D, const RepGeom* __restrict__ geom,
                                          const uint16_t* __restrict__ rep, R h, R r_grid, R rc_min, R rc_max, R ramp,
                                          R* __restrict__ rc) {
  const RepGeom& G = geom[rep[i]];
  auto p = ld_pos<NC>(pos + i);
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

// ---- forces, kick, per-replica thermo -------------------------------------------------
// NC: positions and cell starts through the read-only path (the per-stage
// kernel); the persistent kernel wrote them earlier in its launch and reads
// them with ordinary loads.
// Without EW (the packed loop only): the force alone, no energy, virial or
// pair count (w_i and np_i are not written).
template <typename R, bool TYPED, bool X2, Accum M, bool NC = true, bool EW = true>
__device__ __forceinline__ void b_force(int64_t i, const typename RT<R>::R4* __restrict__ pos,
                                        const R* __restrict__ rc, const int32_t* __restrict__ start,
                                        const ForceArgs<R>& a, const RepGeom* __restrict__ geom,
                                        const uint16_t* __restrict__ rep, typename RT<R>::R4* __restrict__ force,
                                        R* __restrict__ w_i, int32_t* __restrict__ np_i) {
  const RepGeom& G = geom[rep[i]];
  Grid<R> g = rep_cells<R>(G, a.g.edge, a.g.inv_edge, a.g.edge_x, a.g.inv_edge_x);
  double e = 0, w = 0;
  int np = 0;
  force[i] = force_one<R, TYPED, X2, M, NC, EW>(pos, start + G.c0, g, a, (int)i, ld_pos<NC>(pos + i), rc[i], e, w, np);
  if constexpr (EW) {
    w_i[i] = (R)w;
    np_i[i] = np;
  }
}

template <typename R>
__device__ __forceinline__ void b_kick(int64_t i, typename RT<R>::R4* __restrict__ vel,
                                       const typename RT<R>::R4* __restrict__ force, R half_dt,
                                       R* __restrict__ ke_i) {
  auto v = vel[i];
  if (force) {
    auto f = force[i];
    v.x += half_dt * f.x;
    v.y += half_dt * f.y;
    v.z += half_dt * f.z;
    vel[i] = v;
  }
  if (ke_i) ke_i[i] = (R)0.5 * (v.x * v.x + v.y * v.y + v.z * v.z);
}

// Sums (E, W, KE, pairs) of chunk c by the whole block, in FP64 and a fixed
// order, into tpart[q * nchunk + c].
template <typename R>
__device__ __forceinline__ void b_thermo_chunk(int c, const int64_t* __restrict__ chunk, int32_t nchunk,
                                               const typename RT<R>::R4* __restrict__ force,
                                               const R* __restrict__ w_i, const R* __restrict__ ke_i,
                                               const int32_t* __restrict__ np_i, double* __restrict__ tpart) {
  __shared__ double sh[4][32];
  const int64_t p0 = chunk[2 * c], p1 = chunk[2 * c + 1];
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
  __syncthreads();
  if (lane == 0)
    for (int q = 0; q < 4; ++q) sh[q][wid] = v[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[threadIdx.x][k];
    tpart[(int64_t)threadIdx.x * nchunk + c] = t;
  }
}

// thermo[4 r + q] = sum over replica r's chunks, by one warp (lane order fixed).
__device__ __forceinline__ void b_thermo_sum(int r, const int32_t* __restrict__ chunk0, int32_t nchunk,
                                             const double* __restrict__ tpart, double* __restrict__ thermo) {
  const int lane = threadIdx.x & 31;
  const int c0 = chunk0[r], c1 = chunk0[r + 1];
  for (int q = 0; q < 4; ++q) {
    double t = 0;
    for (int c = c0 + lane; c < c1; c += 32) t += tpart[(int64_t)q * nchunk + c];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) thermo[4 * r + q] = t;
  }
}

// The LJ constants of a batch for the force stage (cell edges from params).
template <typename R>
ForceArgs<R> batch_force_args(const dcm_batch* b);

// One timestep (or the initial evaluation) of every replica in a single
// cooperative launch (batch_persist.cu).  drift: half kick and drift before
// binning; recompute: interface, distances and cutoffs after binning; kick:
// the second half kick with the new forces.  Reads buffer s->cur, writes
// buffer 1 - s->cur (the caller flips cur).
template <typename R>
int b_persistent_step(dcm_batch* b, dcm_state* s, R hdt, R dt, bool drift, bool recompute, bool kick,
                      bool energies, cudaStream_t st);
// The accumulation form of the batched force stage (DCM_ACC_FP32,
// DCM_ACC_PLANE_FP64 or DCM_ACC_PLANE_KAHAN).
int batch_accumulation(const dcm_batch* b);
// Size the persistent grid (co-resident blocks) and the work queue; once per batch.
int b_persistent_setup(dcm_batch* b);
// Work items of `tile` particles (a multiple of 32, at most 4096) for the force queue.
int b_persistent_set_tile(dcm_batch* b, int tile);
// Self-test of the bounded grid barrier: one launch of the persistent grid
// whose barrier waits for `phantom` blocks that do not exist, with a wait
// budget of `budget` polls.  Returns DCM_ERR_TIMEOUT (recorded in the device
// status) when the waits run out as they must.
int b_persistent_wait_selftest(dcm_batch* b, int32_t phantom, int64_t budget, cudaStream_t st);

}  // namespace dcm
