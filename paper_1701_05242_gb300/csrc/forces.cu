// Lennard-Jones forces with per-particle cutoffs (Section 2.4, Algorithms 2.2
// and 2.3): i-centric, no Newton's third law, over cell lists.
//
// One thread per particle i in cell-sorted order (a warp therefore covers a
// few neighbouring cells and walks nearly the same neighbour rows).  The
// stencil is culled per particle (Section 2.3's small-bin idea taken to the
// particle level): a row of cells (fixed y, z offset) is visited only if its
// y-z slab lies within rc_i, and only the x-range of cells the sphere of
// radius rc_i actually reaches.  Cells along x are contiguous in the sorted
// order, so every row segment is one contiguous run of j particles.
//
// Periodic images are formed without rounding: an image shifted by -L is
// taken as x_j - L (exact, x_j >= L/2 whenever the pair can be accepted) and
// one shifted by +L as x_i - L on the i side (exact for the same reason), so
// each component r_ij carries a single rounding in FP32.
//
// Pair arithmetic is branch-free: rejected candidates get 1/r^2 = 0, which
// zeroes every term.
#include <algorithm>
#include <cmath>

#include "forces_core.cuh"

namespace dcm {

// Per-warp partial sums of (E, W, pairs): summed across the warp in the
// working precision (32 terms), then stored as one FP64 partial per warp;
// no block barrier, so warps that finish early do not wait.
template <typename R>
__device__ __forceinline__ void warp_partials3(R a, R b, int c, double* part, int64_t nslot) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    part[w] = (double)a;
    part[nslot + w] = (double)b;
    part[2 * nslot + w] = (double)c;
  }
}

template <typename R, bool TYPED>
__global__ void __launch_bounds__(kForceBlock) k_forces(int64_t n, const typename RT<R>::R4* __restrict__ pos,
                                                        const R* __restrict__ rc, const int32_t* __restrict__ start,
                                                        ForceArgs<R> a, typename RT<R>::R4* __restrict__ force,
                                                        double* __restrict__ part, int64_t nwarp) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  R e_out = 0, w_out = 0;
  int np = 0;
  if (i < n) force[i] = force_one<R, TYPED>(pos, start, a.g, a, (int)i, ldg4(pos + i), rc[i], e_out, w_out, np);
  if (part) warp_partials3<R>(e_out, w_out, np, part, nwarp);
}

// ----------------------------------------------------------------------------
// Two-phase force kernel (one type, FP32, eps = sigma = 1): every lane first
// filters its candidates row by row and appends the accepted ones (r_ij and
// r^2) to its own shared-memory buffer; before a row whose window could
// overflow any lane's buffer, and at the end, the warp drains all buffers
// together and only then does the pair arithmetic.  Rejected candidates (about
// two thirds with cell-granular windows) cost a distance test instead of the
// whole pair evaluation.
// ----------------------------------------------------------------------------
constexpr int kBuf = 32;      // accepted pairs buffered per lane
constexpr int kF2Block = 128;

__device__ __forceinline__ void drain(const float4 (*buf)[kF2Block], int cnt, Acc<float>& c) {
  for (int k = 0; k < cnt; ++k) {
    float4 e = buf[k][threadIdx.x];
    float inv = recip(e.w);
    float s6 = inv * inv * inv;
    float pv = s6 * fmaf(2.0f, s6, -1.0f);
    float q = pv * inv;
    c.fx = fmaf(q, e.x, c.fx);
    c.fy = fmaf(q, e.y, c.fy);
    c.fz = fmaf(q, e.z, c.fz);
    c.en += fmaf(s6, s6, -s6);
    c.vir += pv;
  }
  c.np += cnt;
}

template <bool SJ>
__device__ __forceinline__ int filter_range(const float4* __restrict__ pos, int lo, int hi, float xi, float yi,
                                            float zi, float shx, float shy, float shz, float rc2,
                                            float4 (*buf)[kF2Block], int cnt) {
  for (int j = lo; j < hi; ++j) {
    float4 pj = __ldg(pos + j);
    float dx, dy, dz;
    if (SJ) {
      dx = xi - (pj.x + shx);
      dy = yi - (pj.y + shy);
      dz = zi - (pj.z + shz);
    } else {
      dx = xi - pj.x;
      dy = yi - pj.y;
      dz = zi - pj.z;
    }
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < rc2) {
      buf[cnt][threadIdx.x] = make_float4(dx, dy, dz, r2);
      ++cnt;
    }
  }
  return cnt;
}

__global__ void __launch_bounds__(kF2Block) k_forces2(int64_t n, const float4* __restrict__ pos,
                                                      const float* __restrict__ rc, const int32_t* __restrict__ start,
                                                      ForceArgs<float> a, float4* __restrict__ force,
                                                      double* __restrict__ part, int64_t nwarp) {
  __shared__ float4 buf[kBuf][kF2Block];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < n;
  Acc<float> c;
  int cnt = 0;
  float e_out = 0.f, w_out = 0.f;
  const Grid<float>& g = a.g;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const float l = g.edge, il = g.inv_edge;
  float4 pi = live ? __ldg(pos + i) : make_float4(0.f, 0.f, 0.f, 0.f);
  float rci = live ? rc[i] : 0.f;
  if (!(rci <= a.rc_max)) rci = a.rc_max;
  if (!(rci > 0.f)) rci = 0.f;
  const float rc2 = rci * rci;
  const float rc2s = rc2 * 1.000004f;
  const int cx = cell_coord<float>(pi.x, l, il, nx);
  const int cy = cell_coord<float>(pi.y, l, il, ny);
  const int cz = cell_coord<float>(pi.z, l, il, nz);
  const int H = live ? (int)ceilf(rci * il) : -1;
  // the warp walks the union of its lanes' (dz, dy) rows in lockstep
  int Hw = H;
  for (int o = 16; o > 0; o >>= 1) Hw = max(Hw, __shfl_xor_sync(0xffffffffu, Hw, o));
  const int self = (int)i;
  for (int dz = -Hw; dz <= Hw; ++dz) {
    int uz = cz + dz;
    float gz = uz > cz ? (float)uz * l - pi.z : (uz < cz ? pi.z - (float)(uz + 1) * l : 0.f);
    float gz2 = gz * gz;
    int wz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
    float zi = uz >= nz ? pi.z - g.L[2] : pi.z;
    float zsh = uz < 0 ? -g.L[2] : 0.f;
    for (int dy = -Hw; dy <= Hw; ++dy) {
      int uy = cy + dy;
      float gy = uy > cy ? (float)uy * l - pi.y : (uy < cy ? pi.y - (float)(uy + 1) * l : 0.f);
      float gyz2 = gz2 + gy * gy;
      bool on = dz >= -H && dz <= H && dy >= -H && dy <= H && gyz2 < rc2s;
      int ulo = 0, uhi = -1;
      int64_t row = 0;
      float yi = pi.y, ysh = 0.f;
      if (on) {
        int wy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
        yi = uy >= ny ? pi.y - g.L[1] : pi.y;
        ysh = uy < 0 ? -g.L[1] : 0.f;
        float wx = sqrtf(rc2s - gyz2);
        ulo = max((int)floorf((pi.x - wx) * il - 5e-4f), cx - H);
        uhi = min((int)floorf((pi.x + wx) * il + 5e-4f), cx + H);
        row = (int64_t)nx * (wy + (int64_t)ny * wz);
      }
      // the candidates this row can add: the whole window
      int jlo = 0, jhi = 0;
      if (on && ulo <= uhi) {
        int clo = ulo < 0 ? ulo + nx : ulo, chi = uhi >= nx ? uhi - nx : uhi;
        if (ulo >= 0 && uhi < nx) {
          jlo = __ldg(start + row + clo);
          jhi = __ldg(start + row + chi + 1);
        } else {  // wrapped window: count both pieces
          int a0 = __ldg(start + row + clo), a1 = __ldg(start + row + nx);
          int b0 = __ldg(start + row), b1 = __ldg(start + row + chi + 1);
          jlo = 0;
          jhi = (a1 - a0) + (b1 - b0);
        }
      }
      int wlen = jhi - jlo;
      if (__any_sync(0xffffffffu, cnt + wlen > kBuf)) {
        drain(buf, cnt, c);
        cnt = 0;
      }
      if (!on || ulo > uhi) continue;
      if (wlen > kBuf) {
        // a window longer than the buffer (very dense or very wide rows): evaluate in place
        for (int seg = 0; seg < 3; ++seg) {
          int s0, s1;
          float xi = pi.x, xsh = 0.f;
          if (seg == 0) { s0 = ulo; s1 = min(uhi, -1); xsh = -g.L[0]; }
          else if (seg == 1) { s0 = max(ulo, 0); s1 = min(uhi, nx - 1); }
          else { s0 = max(ulo, nx); s1 = uhi; xi = pi.x - g.L[0]; }
          if (s0 > s1) continue;
          int w0 = seg == 0 ? s0 + nx : (seg == 2 ? s0 - nx : s0);
          int w1 = seg == 0 ? s1 + nx : (seg == 2 ? s1 - nx : s1);
          int j0 = __ldg(start + row + w0), j1 = __ldg(start + row + w1 + 1);
          pair_range<float, true, false>(pos, j0, min(j1, self), xi, yi, zi, xsh, ysh, zsh, rc2, 0, a, nullptr, c);
          pair_range<float, true, false>(pos, max(j0, self + 1), j1, xi, yi, zi, xsh, ysh, zsh, rc2, 0, a, nullptr, c);
        }
        continue;
      }
      if (ulo < 0) {
        int s1 = min(uhi, -1);
        cnt = filter_range<true>(pos, __ldg(start + row + ulo + nx), __ldg(start + row + s1 + nx + 1), pi.x, yi, zi,
                                 -g.L[0], ysh, zsh, rc2, buf, cnt);
      }
      {
        int s0 = max(ulo, 0), s1 = min(uhi, nx - 1);
        if (s0 <= s1) {
          int j0 = __ldg(start + row + s0), j1 = __ldg(start + row + s1 + 1);
          if (ysh == 0.f && zsh == 0.f) {
            cnt = filter_range<false>(pos, j0, min(j1, self), pi.x, yi, zi, 0.f, 0.f, 0.f, rc2, buf, cnt);
            cnt = filter_range<false>(pos, max(j0, self + 1), j1, pi.x, yi, zi, 0.f, 0.f, 0.f, rc2, buf, cnt);
          } else {
            cnt = filter_range<true>(pos, j0, j1, pi.x, yi, zi, 0.f, ysh, zsh, rc2, buf, cnt);
          }
        }
      }
      if (uhi >= nx) {
        int s0 = max(ulo, nx);
        cnt = filter_range<true>(pos, __ldg(start + row + s0 - nx), __ldg(start + row + uhi - nx + 1),
                                 pi.x - g.L[0], yi, zi, 0.f, ysh, zsh, rc2, buf, cnt);
      }
    }
  }
  drain(buf, cnt, c);
  if (live) {
    float ush = 0.f;
    if (a.shift) {
      float s2 = 1.f / rc2, s6 = s2 * s2 * s2;
      ush = 4.f * s6 * (s6 - 1.f);
    }
    e_out = 2.f * c.en - 0.5f * (float)c.np * ush;
    w_out = 12.f * c.vir;
    force[i] = make_float4(24.f * c.fx, 24.f * c.fy, 24.f * c.fz, e_out);
  }
  if (part) warp_partials3<float>(e_out, w_out, c.np, part, nwarp);
}

// ----------------------------------------------------------------------------
// Warp-per-particle force kernel (one type, FP32, eps = sigma = 1).
//
// A warp takes one particle i at a time.  Its lanes first cut i's culled
// stencil into pieces (a row window, split where it wraps around the box; at
// most 3 per row) and write them, with running candidate offsets, to shared
// memory.  The flattened candidate sequence is then split into 32 equal
// contiguous blocks, one per lane, so every lane runs the same number of
// iterations.  A candidate j inside rc_i is appended (r_ij, r^2) to the
// warp's ring queue with one ballot; whenever 32 are queued all lanes evaluate
// one pair each, so the pair arithmetic never runs on rejected candidates or
// idle lanes.  All queued pairs belong to i, so the lanes' partial sums are
// simply reduced across the warp at the end.
// ----------------------------------------------------------------------------
constexpr int kWpWarps = 4;        // warps per block
constexpr int kWpMaxHalf = 4;     // stencil half-width in cells (H = ceil(rc / l))
constexpr int kMaxPieces = 3 * (2 * kWpMaxHalf + 1) * (2 * kWpMaxHalf + 1);  // up to 3 pieces a row
constexpr int kQ = 64;             // ring queue per warp

struct Piece {
  int j0;      // first sorted slot
  int len;     // candidates
  int cum;     // candidates before this piece
  int code;    // image code: x 0/1/2, y << 2, z << 4 (1: j - L, 2: i - L)
};

__device__ __forceinline__ void wp_pair(const float4 e, Acc<float>& c) {
  float inv = recip(e.w);
  float s6 = inv * inv * inv;
  float pv = s6 * fmaf(2.0f, s6, -1.0f);
  float q = pv * inv;
  c.fx = fmaf(q, e.x, c.fx);
  c.fy = fmaf(q, e.y, c.fy);
  c.fz = fmaf(q, e.z, c.fz);
  c.en += fmaf(s6, s6, -s6);
  c.vir += pv;
}

__global__ void __launch_bounds__(32 * kWpWarps) k_forces_wp(int64_t n, const float4* __restrict__ pos,
                                                             const float* __restrict__ rc,
                                                             const int32_t* __restrict__ start, ForceArgs<float> a,
                                                             float4* __restrict__ force, double* __restrict__ part) {
  __shared__ Piece pcs[kWpWarps][kMaxPieces];
  __shared__ float4 que[kWpWarps][kQ];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  Piece* P = pcs[wid];
  float4* Q = que[wid];
  const Grid<float>& g = a.g;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const float l = g.edge, il = g.inv_edge;
  const int64_t gw = (int64_t)blockIdx.x * kWpWarps + wid, tw = (int64_t)gridDim.x * kWpWarps;
  double esum = 0.0, wsum = 0.0;  // lane 0's running sums over its particles
  int64_t psum = 0;
  for (int64_t i = gw; i < n; i += tw) {
    const float4 pi = __ldg(pos + i);
    float rci = __ldg(rc + i);
    if (!(rci <= a.rc_max)) rci = a.rc_max;
    if (!(rci > 0.f)) rci = 0.f;
    const float rc2 = rci * rci, rc2s = rc2 * 1.000004f;
    const int cx = cell_coord<float>(pi.x, l, il, nx);
    const int cy = cell_coord<float>(pi.y, l, il, ny);
    const int cz = cell_coord<float>(pi.z, l, il, nz);
    const int H = (int)ceilf(rci * il);
    const int side = 2 * H + 1, nrow = side * side;
    // ---- pieces of the culled stencil, in row order
    int npc = 0, total = 0;
    for (int r0 = 0; r0 < nrow; r0 += 32) {
      int r = r0 + lane;
      // up to three pieces of this row: image -L, no image, image +L in x
      int ja = 0, la = 0, jb = 0, lb = 0, jc = 0, lc = 0, yzc = 0;
      if (r < nrow) {
        int uz = cz - H + r / side, uy = cy - H + r % side;
        float gz = uz > cz ? (float)uz * l - pi.z : (uz < cz ? pi.z - (float)(uz + 1) * l : 0.f);
        float gy = uy > cy ? (float)uy * l - pi.y : (uy < cy ? pi.y - (float)(uy + 1) * l : 0.f);
        float gyz2 = fmaf(gz, gz, gy * gy);
        if (gyz2 < rc2s) {
          int wz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
          int wy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
          yzc = ((uy < 0 ? 1 : (uy >= ny ? 2 : 0)) << 2) | ((uz < 0 ? 1 : (uz >= nz ? 2 : 0)) << 4);
          float wx = sqrtf(rc2s - gyz2);
          int ulo = max(ufloor<float>((pi.x - wx) * il - 5e-4f), cx - H);
          int uhi = min(ufloor<float>((pi.x + wx) * il + 5e-4f), cx + H);
          const int64_t row = (int64_t)nx * (wy + (int64_t)ny * wz);
          if (ulo < 0) {
            int a1 = min(uhi, -1);
            ja = __ldg(start + row + ulo + nx);
            la = __ldg(start + row + a1 + nx + 1) - ja;
          }
          int a0 = max(ulo, 0), a1 = min(uhi, nx - 1);
          if (a0 <= a1) {
            jb = __ldg(start + row + a0);
            lb = __ldg(start + row + a1 + 1) - jb;
          }
          if (uhi >= nx) {
            int c0 = max(ulo, nx);
            jc = __ldg(start + row + c0 - nx);
            lc = __ldg(start + row + uhi - nx + 1) - jc;
          }
        }
      }
      // warp scans of piece counts and candidate counts, then store
      const int cnt = (la > 0) + (lb > 0) + (lc > 0), mylen = la + lb + lc;
      int pcnt = cnt, plsum = mylen;
      for (int o = 1; o < 32; o <<= 1) {
        int t1 = __shfl_up_sync(0xffffffffu, pcnt, o), t2 = __shfl_up_sync(0xffffffffu, plsum, o);
        if (lane >= o) { pcnt += t1; plsum += t2; }
      }
      int k = npc + pcnt - cnt, cb = total + plsum - mylen;
      if (la > 0) { P[k++] = Piece{ja, la, cb, yzc | 1}; cb += la; }
      if (lb > 0) { P[k++] = Piece{jb, lb, cb, yzc}; cb += lb; }
      if (lc > 0) P[k] = Piece{jc, lc, cb, yzc | 2};
      npc += __shfl_sync(0xffffffffu, pcnt, 31);
      total += __shfl_sync(0xffffffffu, plsum, 31);
    }
    __syncwarp();
    // ---- each lane: a contiguous block of the flattened candidates
    const int S = (total + 31) >> 5;
    int c = lane * S, cend = min(total, c + S);
    // first piece of the block: binary search on cum
    int lo = 0, hi = npc - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (P[mid].cum <= c) lo = mid; else hi = mid - 1;
    }
    int pk = lo;
    Piece cur = npc > 0 ? P[pk] : Piece{0, 0, 0, 0};
    float xi = pi.x, yi = pi.y, zi = pi.z, sx = 0.f, sy = 0.f, sz = 0.f;
    auto set_frame = [&](int code) {
      int xc = code & 3, yc = (code >> 2) & 3, zc = code >> 4;
      xi = xc == 2 ? pi.x - g.L[0] : pi.x;
      yi = yc == 2 ? pi.y - g.L[1] : pi.y;
      zi = zc == 2 ? pi.z - g.L[2] : pi.z;
      sx = xc == 1 ? -g.L[0] : 0.f;
      sy = yc == 1 ? -g.L[1] : 0.f;
      sz = zc == 1 ? -g.L[2] : 0.f;
    };
    set_frame(cur.code);
    Acc<float> acc;
    int head = 0, tail = 0;  // ring queue indices (warp-uniform)
    for (int t = 0; t < S; ++t, ++c) {
      bool ok = c < cend;
      if (ok && c >= cur.cum + cur.len) {
        do { cur = P[++pk]; } while (c >= cur.cum + cur.len);
        set_frame(cur.code);
      }
      bool take = false;
      float4 e;
      if (ok) {
        int j = cur.j0 + (c - cur.cum);
        float4 pj = __ldg(pos + j);
        e.x = xi - (pj.x + sx);
        e.y = yi - (pj.y + sy);
        e.z = zi - (pj.z + sz);
        e.w = fmaf(e.x, e.x, fmaf(e.y, e.y, e.z * e.z));
        take = e.w < rc2 && !(j == (int)i && cur.code == 0);
      }
      unsigned m = __ballot_sync(0xffffffffu, take);
      if (take) Q[(tail + __popc(m & lt)) & (kQ - 1)] = e;
      tail += __popc(m);
      if (tail - head >= 32) {
        __syncwarp();
        wp_pair(Q[(head + lane) & (kQ - 1)], acc);
        head += 32;
        acc.np += 1;
        __syncwarp();
      }
    }
    __syncwarp();
    if (lane < tail - head) {
      wp_pair(Q[(head + lane) & (kQ - 1)], acc);
      acc.np += 1;
    }
    __syncwarp();
    // ---- reduce the lanes' partial sums of particle i
    for (int o = 16; o > 0; o >>= 1) {
      acc.fx += __shfl_xor_sync(0xffffffffu, acc.fx, o);
      acc.fy += __shfl_xor_sync(0xffffffffu, acc.fy, o);
      acc.fz += __shfl_xor_sync(0xffffffffu, acc.fz, o);
      acc.en += __shfl_xor_sync(0xffffffffu, acc.en, o);
      acc.vir += __shfl_xor_sync(0xffffffffu, acc.vir, o);
      acc.np += __shfl_xor_sync(0xffffffffu, acc.np, o);
    }
    float ush = 0.f;
    if (a.shift && rc2 > 0.f) {
      float s2 = 1.f / rc2, s6 = s2 * s2 * s2;
      ush = 4.f * s6 * (s6 - 1.f);
    }
    float e_i = 2.f * acc.en - 0.5f * (float)acc.np * ush;
    float w_i = 12.f * acc.vir;
    if (lane == 0) force[i] = make_float4(24.f * acc.fx, 24.f * acc.fy, 24.f * acc.fz, e_i);
    esum += (double)e_i;
    wsum += (double)w_i;
    psum += acc.np;
    __syncwarp();
  }
  if (part && lane == 0) {
    part[gw] = esum;
    part[tw + gw] = wsum;
    part[2 * tw + gw] = (double)psum;
  }
}

// Kernels 2 and 3 serve one-type mixed-precision runs with eps = sigma = 1;
// kernel 3's piece table holds stencils of up to 9 x 9 rows.
int resolve_force_kernel(const dcm_ctx* ctx) {
  int k = force_kernel_choice(ctx->p);
  if (k == DCM_FORCE_THREAD) return k;
  if (ctx->p.precision != DCM_PREC_MIXED || lj_general(lj_table(ctx->p))) return DCM_FORCE_THREAD;
  if (k == DCM_FORCE_WARP && std::ceil(ctx->p.rc_max / ctx->p.l) > (double)kWpMaxHalf) return DCM_FORCE_THREAD;
  return k;
}

template <typename R>
int lj_forces(dcm_ctx* ctx, int64_t n, const typename RT<R>::R4* pos, const R* rc, const int32_t* cell_start,
              typename RT<R>::R4* force, double* totals, cudaStream_t st) {
  if (n <= 0) {
    if (totals) DCM_CUDA_TRY(ctx, cudaMemsetAsync(totals, 0, 3 * sizeof(double), st));
    return DCM_OK;
  }
  ForceArgs<R> a;
  a.g = cell_grid<R>(ctx);
  LJTable t = lj_table(ctx->p);
  a.ntypes = t.ntypes;
  for (int k = 0; k < 16; ++k) {
    a.eps24[k] = (R)t.deps24[k];
    a.eps4[k] = (R)t.deps4[k];
    a.sig2[k] = (R)t.dsig2[k];
  }
  a.shift = ctx->p.shift_energy;
  a.rc_max = (R)ctx->p.rc_max;
  int64_t nblk = (n + kForceBlock - 1) / kForceBlock;
  int64_t nwarp = nblk * (kForceBlock / 32);
  if (totals && nwarp > ctx->red_cap)
    return set_error(ctx, DCM_ERR_CAPACITY, "force reduction needs %lld partials", (long long)nwarp);
  double* part = totals ? ctx->red : nullptr;
  auto kern = lj_general(t) ? k_forces<R, true> : k_forces<R, false>;
  stage_begin(ctx, DCM_STAGE_FORCES, st);
  bool done = false;
  if constexpr (sizeof(R) == 4) {
    const ForceArgs<float>& af = a;
    if (resolve_force_kernel(ctx) == DCM_FORCE_WARP) {
      // a grid of 16 waves of blocks strides over the particles
      int64_t nblk_wp = std::min<int64_t>((n + kWpWarps - 1) / kWpWarps, (int64_t)152 * 16 * 4);
      if (totals) nblk_wp = std::min<int64_t>(nblk_wp, ctx->red_cap / kWpWarps);
      DCM_LAUNCH(ctx, k_forces_wp, (unsigned)nblk_wp, 32 * kWpWarps, 0, st, n, pos, rc, cell_start, af, force, part);
      nwarp = nblk_wp * kWpWarps;
      done = true;
    } else if (resolve_force_kernel(ctx) == DCM_FORCE_TWO_PHASE) {
      static_assert(kF2Block == kForceBlock, "partials layout assumes equal blocks");
      DCM_LAUNCH(ctx, k_forces2, (unsigned)nblk, kF2Block, 0, st, n, pos, rc, cell_start, af, force, part, nwarp);
      done = true;
    }
  }
  if (!done) DCM_LAUNCH(ctx, kern, (unsigned)nblk, kForceBlock, 0, st, n, pos, rc, cell_start, a, force, part, nwarp);
  stage_end(ctx, DCM_STAGE_FORCES, st);
  int r = check_launch(ctx, "lj_forces");
  if (r) return r;
  if (totals) return reduce_partials(ctx, part, nwarp, 3, totals, false, st);
  return DCM_OK;
}

template int lj_forces<float>(dcm_ctx*, int64_t, const float4*, const float*, const int32_t*, float4*, double*,
                              cudaStream_t);
template int lj_forces<double>(dcm_ctx*, int64_t, const dvec4*, const double*, const int32_t*, dvec4*, double*,
                               cudaStream_t);

}  // namespace dcm
