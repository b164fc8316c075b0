/*
 * FP64 CPU oracle for the Dynamic Cutoff Method's per-timestep path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code with the CUDA implementation.
 *
 * Everything is plain, sequential, double precision and written for checking
 * by eye against the paper (Springer, Ismail, Bientinesi, "A Scalable,
 * Linear-Time Dynamic Cutoff Algorithm for Molecular Dynamics"):
 *   - binning into linked cells (Sections 2.1 and 2.3),
 *   - gray-scale density volume, two-phase segmentation and interface boxes
 *     (Section 2.1, Eq. 4),
 *   - cutoff-based fast sweeping (Section 2.2, Algorithm 2.1) plus Jacobi and
 *     Gauss-Seidel sweeps used as independent checks,
 *   - trilinear particle-interface distance and cutoff rule (Section 2.2),
 *   - i-centric Lennard-Jones forces without Newton's third law (Section 2.4,
 *     Algorithms 2.2 and 2.3), both O(N^2) and over cells,
 *   - velocity Verlet (Section 2),
 *   - the adjoint of a loss on forces and energy (extension; see below).
 * Inputs are FP32 values widened exactly to double by the caller.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Binning (Section 2.1: particles binned into boxes; Section 2.3: linked    */
/* cells).  Cell of coordinate x is the exact floor(x / l), clamped to       */
/* [0, n-1].  l has a short mantissa (checked by the caller), so k*l is      */
/* exact in double and the correction loop makes the floor exact.            */
/* ------------------------------------------------------------------------ */
int64_t orc_cell_coord(double x, double l, int64_t n) {
  if (!(x >= 0.0)) return 0;               /* negative or NaN: first cell */
  if (!(x < (double)n * l)) return n - 1;  /* beyond the box or +inf: last cell */
  double q = floor(x / l);
  if (q * l > x) q -= 1.0;                 /* x / l is within one unit of the quotient */
  else if ((q + 1.0) * l <= x) q += 1.0;
  int64_t k = (int64_t)q;
  if (k < 0) k = 0;
  if (k > n - 1) k = n - 1;
  return k;
}

int64_t orc_cell_of(const double* p, const double* l, const int64_t* nc) {
  int64_t cx = orc_cell_coord(p[0], l[0], nc[0]);
  int64_t cy = orc_cell_coord(p[1], l[1], nc[1]);
  int64_t cz = orc_cell_coord(p[2], l[2], nc[2]);
  return cx + nc[0] * (cy + nc[1] * cz);
}

/* Stable counting sort of particles by cell.  cell[i]: cell of input particle
 * i; count[c]; start[c] = exclusive prefix sum (start[ncell] = n); perm[k]:
 * input index of the particle in sorted slot k (ties kept in input order). */
void orc_bin(int64_t n, const double* pos, const double* l, const int64_t* nc, int32_t* cell,
             int32_t* count, int32_t* start, int32_t* perm) {
  int64_t ncell = nc[0] * nc[1] * nc[2];
  for (int64_t c = 0; c < ncell; ++c) count[c] = 0;
  for (int64_t i = 0; i < n; ++i) {
    cell[i] = (int32_t)orc_cell_of(pos + 3 * i, l, nc);
    count[cell[i]]++;
  }
  int64_t run = 0;
  for (int64_t c = 0; c < ncell; ++c) {
    start[c] = (int32_t)run;
    run += count[c];
  }
  start[ncell] = (int32_t)run;
  int32_t* fill = (int32_t*)calloc((size_t)ncell, sizeof(int32_t));
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = cell[i];
    perm[start[c] + fill[c]] = (int32_t)i;
    fill[c]++;
  }
  free(fill);
}

/* ------------------------------------------------------------------------ */
/* Interface detection (Section 2.1, Eq. 4).                                 */
/* ------------------------------------------------------------------------ */
static int64_t wrap(int64_t k, int64_t n) {
  k %= n;
  return k < 0 ? k + n : k;
}

/* Gray-scale volume: box sum of particle counts over the (2w+1)^3 periodic
 * neighbourhood of every box (plain definition, one box at a time). */
void orc_smooth(const int32_t* count, const int64_t* nh, int w, int32_t* g) {
  for (int64_t z = 0; z < nh[2]; ++z)
    for (int64_t y = 0; y < nh[1]; ++y)
      for (int64_t x = 0; x < nh[0]; ++x) {
        int64_t s = 0;
        for (int c = -w; c <= w; ++c)
          for (int b = -w; b <= w; ++b)
            for (int a = -w; a <= w; ++a)
              s += count[wrap(x + a, nh[0]) + nh[0] * (wrap(y + b, nh[1]) + nh[1] * wrap(z + c, nh[2]))];
        g[x + nh[0] * (y + nh[1] * z)] = (int32_t)s;
      }
}

/* Two-phase segmentation without the length term: with phase means c0 < c1
 * fixed, the minimiser of the piecewise-constant two-phase functional is the
 * threshold at (c0 + c1) / 2; alternating means and threshold is 2-means.
 * Integer form: s = (g >= T), T = floor(midpoint) + 1.  Returns T; if one
 * phase is empty the volume has no interface and T = g_max + 1. */
int64_t orc_two_means(const int32_t* g, int64_t nbox, int max_iter) {
  int64_t gmin = g[0], gmax = g[0];
  for (int64_t b = 1; b < nbox; ++b) {
    if (g[b] < gmin) gmin = g[b];
    if (g[b] > gmax) gmax = g[b];
  }
  int64_t T = (gmin + gmax) / 2;
  for (int it = 0; it < max_iter; ++it) {
    int64_t n0 = 0, n1 = 0, s0 = 0, s1 = 0;
    for (int64_t b = 0; b < nbox; ++b) {
      if (g[b] < T) {
        n0++;
        s0 += g[b];
      } else {
        n1++;
        s1 += g[b];
      }
    }
    if (n0 == 0 || n1 == 0) return gmax + 1;
    int64_t Tn = (s0 * n1 + s1 * n0) / (2 * n0 * n1) + 1;
    if (Tn == T) break;
    T = Tn;
  }
  return T;
}

/* Segmented volume S (Eq. 4) and interface boxes: a box is at the interface if
 * it is in the high-density phase and one of its six face neighbours is not. */
void orc_segment(const int32_t* g, const int64_t* nh, int64_t T, uint8_t* s, uint8_t* iface) {
  int64_t nbox = nh[0] * nh[1] * nh[2];
  for (int64_t b = 0; b < nbox; ++b) s[b] = g[b] >= T ? 1 : 0;
  for (int64_t z = 0; z < nh[2]; ++z)
    for (int64_t y = 0; y < nh[1]; ++y)
      for (int64_t x = 0; x < nh[0]; ++x) {
        int64_t b = x + nh[0] * (y + nh[1] * z);
        int f = 0;
        if (s[b]) {
          f |= !s[wrap(x - 1, nh[0]) + nh[0] * (y + nh[1] * z)];
          f |= !s[wrap(x + 1, nh[0]) + nh[0] * (y + nh[1] * z)];
          f |= !s[x + nh[0] * (wrap(y - 1, nh[1]) + nh[1] * z)];
          f |= !s[x + nh[0] * (wrap(y + 1, nh[1]) + nh[1] * z)];
          f |= !s[x + nh[0] * (y + nh[1] * wrap(z - 1, nh[2]))];
          f |= !s[x + nh[0] * (y + nh[1] * wrap(z + 1, nh[2]))];
        }
        iface[b] = (uint8_t)f;
      }
}

/* Interface boxes of a given segmented volume S: high-density boxes with a
 * low-density face neighbour (the same rule as orc_segment). */
void orc_interface(const uint8_t* s, const int64_t* nh, uint8_t* iface) {
  for (int64_t z = 0; z < nh[2]; ++z)
    for (int64_t y = 0; y < nh[1]; ++y)
      for (int64_t x = 0; x < nh[0]; ++x) {
        int64_t b = x + nh[0] * (y + nh[1] * z);
        int f = 0;
        if (s[b]) {
          f |= !s[wrap(x - 1, nh[0]) + nh[0] * (y + nh[1] * z)];
          f |= !s[wrap(x + 1, nh[0]) + nh[0] * (y + nh[1] * z)];
          f |= !s[x + nh[0] * (wrap(y - 1, nh[1]) + nh[1] * z)];
          f |= !s[x + nh[0] * (wrap(y + 1, nh[1]) + nh[1] * z)];
          f |= !s[x + nh[0] * (y + nh[1] * wrap(z - 1, nh[2]))];
          f |= !s[x + nh[0] * (y + nh[1] * wrap(z + 1, nh[2]))];
        }
        iface[b] = (uint8_t)f;
      }
}

/* Regularised two-phase segmentation (Section 2.1: the piecewise constant
 * Mumford-Shah functional for two-phase segmentation, refs. [1, 18]).
 * Reading: on the periodic grid of box counts g the functional of a binary
 * volume s with phase values c0 (low density) and c1 (high density) is
 *   E(s; c0, c1) = sum_b [ s_b (g_b - c1)^2 + (1 - s_b) (g_b - c0)^2 ]
 *                + nu sum over box faces |s_b - s_b'|
 * (the length term counts the faces between the phases).  It is minimised by
 * alternating the phase values (the means of g over each phase) with the
 * minimisation over s for fixed values.  For fixed values E is, up to a
 * constant, sum_b w_b s_b + nu sum |D s| with w_b = (g_b - c1)^2 - (g_b - c0)^2;
 * its convex relaxation over u in [0, 1]^n (the face sum is a total variation
 * on the grid graph) has binary minimisers given by thresholding any
 * minimiser at 1/2, and is solved by the first-order primal-dual iteration of
 * Chambolle and Pock (2011), a stencil on the grid:
 *   p_f  <- clip(p_f + sigma (D ubar)_f, -nu, nu)         (one p per face)
 *   u'_b <- clip(u_b - tau ((D^T p)_b + w_b), 0, 1)
 *   ubar <- 2 u' - u,  u <- u'
 * with (D u)_f = u_{b+e} - u_b for the face f between b and b + e, and
 * (D^T p)_b = sum_e (p_{b-e, e} - p_{b, e}); tau = sigma = 0.28 (tau sigma
 * ||D||^2 < 1, ||D||^2 <= 12 on the 3D grid).  Each outer iteration starts
 * from u = s, p = 0, runs `inner` iterations and sets s_b = (u_b >= 1/2); the
 * loop stops after `outer` iterations, when s no longer changes, or when a
 * phase is empty (s then stays as it is).  s is the initial volume on input
 * and the result on output; u (nullable) receives the last relaxed solution
 * and c[0..1] the phase values of the last outer iteration.  Returns the
 * number of outer iterations run. */
int orc_ms_segment(const int32_t* g, const int64_t* nh, double nu, int inner, int outer, uint8_t* s, double* u_out,
                   double* c) {
  const int64_t nx = nh[0], ny = nh[1], nz = nh[2], nbox = nx * ny * nz;
  const double tau = 0.28, sigma = 0.28;
  double* w = (double*)malloc(sizeof(double) * (size_t)nbox);
  double* u = (double*)malloc(sizeof(double) * (size_t)nbox);
  double* ub = (double*)malloc(sizeof(double) * (size_t)nbox);
  double* p = (double*)malloc(sizeof(double) * 3 * (size_t)nbox); /* p[3 b + e]: face between b and b + e */
  int done = 0;
  for (int o = 0; o < outer; ++o) {
    /* phase values: the means of g over each phase */
    double s0 = 0.0, s1 = 0.0;
    int64_t n0 = 0, n1 = 0;
    for (int64_t b = 0; b < nbox; ++b) {
      if (s[b]) {
        s1 += g[b];
        ++n1;
      } else {
        s0 += g[b];
        ++n0;
      }
    }
    if (n0 == 0 || n1 == 0) break;
    const double c0 = s0 / (double)n0, c1 = s1 / (double)n1;
    if (c) {
      c[0] = c0;
      c[1] = c1;
    }
    for (int64_t b = 0; b < nbox; ++b) {
      w[b] = (g[b] - c1) * (g[b] - c1) - (g[b] - c0) * (g[b] - c0);
      u[b] = s[b] ? 1.0 : 0.0;
      ub[b] = u[b];
      p[3 * b] = p[3 * b + 1] = p[3 * b + 2] = 0.0;
    }
    for (int it = 0; it < inner; ++it) {
      /* dual step on every face (b, b + e) */
      for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
          for (int64_t x = 0; x < nx; ++x) {
            const int64_t b = x + nx * (y + ny * z);
            const int64_t nb[3] = {wrap(x + 1, nx) + nx * (y + ny * z), x + nx * (wrap(y + 1, ny) + ny * z),
                                   x + nx * (y + ny * wrap(z + 1, nz))};
            for (int e = 0; e < 3; ++e) {
              double q = p[3 * b + e] + sigma * (ub[nb[e]] - ub[b]);
              p[3 * b + e] = q < -nu ? -nu : (q > nu ? nu : q);
            }
          }
      /* primal step on every box */
      for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
          for (int64_t x = 0; x < nx; ++x) {
            const int64_t b = x + nx * (y + ny * z);
            const int64_t pb[3] = {wrap(x - 1, nx) + nx * (y + ny * z), x + nx * (wrap(y - 1, ny) + ny * z),
                                   x + nx * (y + ny * wrap(z - 1, nz))};
            double dtp = 0.0;
            for (int e = 0; e < 3; ++e) dtp += p[3 * pb[e] + e] - p[3 * b + e];
            double v = u[b] - tau * (dtp + w[b]);
            v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
            ub[b] = 2.0 * v - u[b];
            u[b] = v;
          }
    }
    ++done;
    int changed = 0;
    for (int64_t b = 0; b < nbox; ++b) {
      const uint8_t t = u[b] >= 0.5 ? 1 : 0;
      changed |= t != s[b];
      s[b] = t;
    }
    if (u_out)
      for (int64_t b = 0; b < nbox; ++b) u_out[b] = u[b];
    if (!changed) break;
  }
  free(w);
  free(u);
  free(ub);
  free(p);
  return done;
}

/* Removal of small connected components (Section 2.1: "bubbles" of either
 * phase inside the other are filtered out by volume; the filter itself is in
 * the paper's reference [25], not available).  Reading: components are sets
 * of boxes of equal S joined through faces (6-connectivity, periodic); every
 * component of fewer than min_boxes boxes, of either phase, takes the other
 * value; all components are found on the input volume and flipped together.
 * Plain breadth-first search.  Returns the number of flipped components. */
int64_t orc_remove_small_components(const uint8_t* s_in, const int64_t* nh, int64_t min_boxes, uint8_t* s_out) {
  int64_t nbox = nh[0] * nh[1] * nh[2];
  int64_t* comp = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbox);
  int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbox);
  for (int64_t b = 0; b < nbox; ++b) comp[b] = -1;
  int64_t flipped = 0;
  for (int64_t seed = 0; seed < nbox; ++seed) {
    if (comp[seed] >= 0) continue;
    /* breadth-first search from the seed over equal-valued face neighbours */
    int64_t head = 0, tail = 0;
    queue[tail++] = seed;
    comp[seed] = seed;
    while (head < tail) {
      int64_t b = queue[head++];
      int64_t x = b % nh[0], y = (b / nh[0]) % nh[1], z = b / (nh[0] * nh[1]);
      int64_t nb[6] = {wrap(x - 1, nh[0]) + nh[0] * (y + nh[1] * z), wrap(x + 1, nh[0]) + nh[0] * (y + nh[1] * z),
                       x + nh[0] * (wrap(y - 1, nh[1]) + nh[1] * z), x + nh[0] * (wrap(y + 1, nh[1]) + nh[1] * z),
                       x + nh[0] * (y + nh[1] * wrap(z - 1, nh[2])), x + nh[0] * (y + nh[1] * wrap(z + 1, nh[2]))};
      for (int k = 0; k < 6; ++k)
        if (comp[nb[k]] < 0 && s_in[nb[k]] == s_in[seed]) {
          comp[nb[k]] = seed;
          queue[tail++] = nb[k];
        }
    }
    /* the queue now holds exactly this component (tail boxes) */
    int flip = tail < min_boxes;
    flipped += flip;
    for (int64_t q = 0; q < tail; ++q) s_out[queue[q]] = (uint8_t)(flip ? !s_in[seed] : s_in[seed]);
  }
  free(comp);
  free(queue);
  return flipped;
}

/* ------------------------------------------------------------------------ */
/* Box-interface distances (Section 2.2).                                    */
/* ------------------------------------------------------------------------ */
/* Local fast-sweeping update of one box (Zhao's Godunov upwind discretisation
 * of |grad d| = 1 on spacing h): a_k = smaller of the two axis-k neighbours,
 * sorted a1 <= a2 <= a3; the candidate is the 1-, 2- or 3-neighbour solution,
 * and the box keeps the smaller of its value and the candidate. */
static double godunov(const double* D, const int64_t* nh, int64_t x, int64_t y, int64_t z, double h) {
  double a[3];
  a[0] = fmin(D[wrap(x - 1, nh[0]) + nh[0] * (y + nh[1] * z)], D[wrap(x + 1, nh[0]) + nh[0] * (y + nh[1] * z)]);
  a[1] = fmin(D[x + nh[0] * (wrap(y - 1, nh[1]) + nh[1] * z)], D[x + nh[0] * (wrap(y + 1, nh[1]) + nh[1] * z)]);
  a[2] = fmin(D[x + nh[0] * (y + nh[1] * wrap(z - 1, nh[2]))], D[x + nh[0] * (y + nh[1] * wrap(z + 1, nh[2]))]);
  /* sort ascending */
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2 - i; ++j)
      if (a[j] > a[j + 1]) {
        double t = a[j];
        a[j] = a[j + 1];
        a[j + 1] = t;
      }
  double d = a[0] + h;
  if (d > a[1]) {
    d = 0.5 * (a[0] + a[1] + sqrt(2.0 * h * h - (a[0] - a[1]) * (a[0] - a[1])));
    if (d > a[2]) {
      double sa = a[0] + a[1] + a[2];
      double sq = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
      d = (sa + sqrt(sa * sa - 3.0 * (sq - h * h))) / 3.0;
    }
  }
  double cur = D[x + nh[0] * (y + nh[1] * z)];
  return d < cur ? d : cur;
}

/* Initial distances (Algorithm 2.1, initialize): 0 at interface boxes and in
 * the low-density phase, +inf in the high-density phase. */
void orc_distance_init(const uint8_t* s, const uint8_t* iface, int64_t nbox, double* D) {
  for (int64_t b = 0; b < nbox; ++b) D[b] = (!s[b] || iface[b]) ? 0.0 : INFINITY;
}

/* Cutoff-based fast sweeping, Algorithm 2.1, on one process (no ghost
 * exchange; periodic neighbours are local).  Q starts with the boxes adjacent
 * to the interface that have non-zero distance; each pass processes Q
 * breadth-first, accepts an updated distance only if it is <= r_grid, records
 * the largest change and queues the six neighbours of every accepted box.
 * Readings: the local FSM update keeps min(current, candidate); the change
 * tolerance epsilon tends to 0, i.e. the loop stops after the first pass that
 * changes no box.  Returns the number of passes, or -1 if iter_max passes did
 * not converge. */
int orc_cfsm(const uint8_t* s, const uint8_t* iface, const int64_t* nh, double h, double r_grid,
             int iter_max, double* D) {
  int64_t nbox = nh[0] * nh[1] * nh[2];
  orc_distance_init(s, iface, nbox, D);
  int64_t* Q = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbox);
  int64_t* Qn = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbox);
  uint8_t* inq = (uint8_t*)calloc((size_t)nbox, 1);
  int64_t nq = 0, nqn = 0;
  /* initialize(D, Q): boxes with non-zero distance next to a zero-distance box */
  for (int64_t z = 0; z < nh[2]; ++z)
    for (int64_t y = 0; y < nh[1]; ++y)
      for (int64_t x = 0; x < nh[0]; ++x) {
        int64_t b = x + nh[0] * (y + nh[1] * z);
        if (D[b] == 0.0) continue;
        int64_t nb[6] = {wrap(x - 1, nh[0]) + nh[0] * (y + nh[1] * z), wrap(x + 1, nh[0]) + nh[0] * (y + nh[1] * z),
                         x + nh[0] * (wrap(y - 1, nh[1]) + nh[1] * z), x + nh[0] * (wrap(y + 1, nh[1]) + nh[1] * z),
                         x + nh[0] * (y + nh[1] * wrap(z - 1, nh[2])), x + nh[0] * (y + nh[1] * wrap(z + 1, nh[2]))};
        for (int k = 0; k < 6; ++k)
          if (D[nb[k]] == 0.0 && iface[nb[k]]) {
            Q[nq++] = b;
            inq[b] = 1;
            break;
          }
      }
  int iter = 0, converged = 0;
  for (iter = 0; iter < iter_max; ++iter) {
    double de = 0.0;
    memset(inq, 0, (size_t)nbox);
    nqn = 0;
    for (int64_t qi = 0; qi < nq; ++qi) {
      int64_t b = Q[qi];
      int64_t x = b % nh[0], y = (b / nh[0]) % nh[1], z = b / (nh[0] * nh[1]);
      double dn = godunov(D, nh, x, y, z, h);
      if (dn <= r_grid) {
        double ch = fabs(D[b] - dn);
        if (ch > de) de = ch;
        D[b] = dn;
        int64_t nb[6] = {wrap(x - 1, nh[0]) + nh[0] * (y + nh[1] * z), wrap(x + 1, nh[0]) + nh[0] * (y + nh[1] * z),
                         x + nh[0] * (wrap(y - 1, nh[1]) + nh[1] * z), x + nh[0] * (wrap(y + 1, nh[1]) + nh[1] * z),
                         x + nh[0] * (y + nh[1] * wrap(z - 1, nh[2])), x + nh[0] * (y + nh[1] * wrap(z + 1, nh[2]))};
        for (int k = 0; k < 6; ++k)
          if (D[nb[k]] != 0.0 && !inq[nb[k]]) {
            inq[nb[k]] = 1;
            Qn[nqn++] = nb[k];
          }
      }
    }
    /* swapQueues, emptyQueue */
    int64_t* t = Q;
    Q = Qn;
    Qn = t;
    nq = nqn;
    if (!(de > 0.0)) {
      converged = 1;
      ++iter;
      break;
    }
  }
  free(Q);
  free(Qn);
  free(inq);
  return converged ? iter : -1;
}

/* Independent check 1: Jacobi iteration of the same local update over every
 * box (all boxes read the previous iterate), accepting values <= r_grid,
 * until no box changes.  Returns the number of sweeps or -1. */
int orc_distance_jacobi(const uint8_t* s, const uint8_t* iface, const int64_t* nh, double h,
                        double r_grid, int iter_max, double* D) {
  int64_t nbox = nh[0] * nh[1] * nh[2];
  orc_distance_init(s, iface, nbox, D);
  double* Dn = (double*)malloc(sizeof(double) * (size_t)nbox);
  int it;
  for (it = 0; it < iter_max; ++it) {
    int changed = 0;
    for (int64_t z = 0; z < nh[2]; ++z)
      for (int64_t y = 0; y < nh[1]; ++y)
        for (int64_t x = 0; x < nh[0]; ++x) {
          int64_t b = x + nh[0] * (y + nh[1] * z);
          double dn = godunov(D, nh, x, y, z, h);
          Dn[b] = (dn <= r_grid) ? dn : D[b];
          if (Dn[b] != D[b]) changed = 1;
        }
    memcpy(D, Dn, sizeof(double) * (size_t)nbox);
    if (!changed) break;
  }
  free(Dn);
  return it < iter_max ? it + 1 : -1;
}

/* Independent check 2: Gauss-Seidel sweeps in Zhao's eight alternating
 * orderings (x, y, z each ascending or descending), updated in place. */
int orc_distance_sweep8(const uint8_t* s, const uint8_t* iface, const int64_t* nh, double h,
                        double r_grid, int iter_max, double* D) {
  int64_t nbox = nh[0] * nh[1] * nh[2];
  orc_distance_init(s, iface, nbox, D);
  int it;
  for (it = 0; it < iter_max; ++it) {
    int changed = 0;
    for (int o = 0; o < 8; ++o) {
      int sx = (o & 1) ? -1 : 1, sy = (o & 2) ? -1 : 1, sz = (o & 4) ? -1 : 1;
      for (int64_t kz = 0; kz < nh[2]; ++kz) {
        int64_t z = sz > 0 ? kz : nh[2] - 1 - kz;
        for (int64_t ky = 0; ky < nh[1]; ++ky) {
          int64_t y = sy > 0 ? ky : nh[1] - 1 - ky;
          for (int64_t kx = 0; kx < nh[0]; ++kx) {
            int64_t x = sx > 0 ? kx : nh[0] - 1 - kx;
            int64_t b = x + nh[0] * (y + nh[1] * z);
            double dn = godunov(D, nh, x, y, z, h);
            if (dn <= r_grid && dn != D[b]) {
              D[b] = dn;
              changed = 1;
            }
          }
        }
      }
    }
    if (!changed) break;
  }
  return it < iter_max ? it + 1 : -1;
}

/* ------------------------------------------------------------------------ */
/* Cutoff assignment (Section 2.2): particle-interface distance delta_i by   */
/* trilinear interpolation of min(D, r_grid) between box centres (k + 1/2)h  */
/* (periodic), then rc = clamp(rc_max - (rc_max - rc_min) delta/ramp).       */
/* ------------------------------------------------------------------------ */
double orc_interp_distance(const double* p, const double* D, const int64_t* nh, double h, double r_grid) {
  int64_t k[3];
  double t[3];
  for (int d = 0; d < 3; ++d) {
    double u = p[d] / h - 0.5;
    double f = isfinite(u) ? floor(u) : 0.0;
    /* exact floor of (x - h/2) / h: (f + 1/2) h is exact for short-mantissa h */
    if ((f + 0.5) * h > p[d]) f -= 1.0;
    else if ((f + 1.5) * h <= p[d]) f += 1.0;
    k[d] = (int64_t)f;
    t[d] = (p[d] - (f + 0.5) * h) / h;
  }
  double acc = 0.0;
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        int64_t bx = wrap(k[0] + a, nh[0]), by = wrap(k[1] + b, nh[1]), bz = wrap(k[2] + c, nh[2]);
        double v = D[bx + nh[0] * (by + nh[1] * bz)];
        if (v > r_grid) v = r_grid;
        double w = (a ? t[0] : 1.0 - t[0]) * (b ? t[1] : 1.0 - t[1]) * (c ? t[2] : 1.0 - t[2]);
        acc += w * v;
      }
  return acc;
}

double orc_cutoff_rule(double delta, double rc_min, double rc_max, double ramp) {
  if (!(ramp > 0.0)) return delta > 0.0 ? rc_min : rc_max; /* step: no ramp */
  double rc = rc_max - (rc_max - rc_min) * delta / ramp;
  if (rc < rc_min) rc = rc_min;
  if (rc > rc_max) rc = rc_max;
  return rc;
}

void orc_cutoffs(int64_t n, const double* pos, const double* D, const int64_t* nh, double h,
                 double r_grid, double rc_min, double rc_max, double ramp, double* delta, double* rc) {
  for (int64_t i = 0; i < n; ++i) {
    double di = orc_interp_distance(pos + 3 * i, D, nh, h, r_grid);
    if (delta) delta[i] = di;
    rc[i] = orc_cutoff_rule(di, rc_min, rc_max, ramp);
  }
}

/* ------------------------------------------------------------------------ */
/* Forces (Section 2.4, Algorithms 2.2/2.3).                                 */
/* Pair rule: j contributes to i iff j != i and |r_ij| < rc[i] (strict), with */
/* r_ij = r_i - r_j the minimum image.  No Newton's third law: f_j is never  */
/* updated from i's loop.  Lennard-Jones 12-6 with Lorentz-Berthelot mixing: */
/* U(r) = 4 eps [(s/r)^12 - (s/r)^6], F_i += 24 eps [2(s/r)^12 - (s/r)^6]/r^2 */
/* r_ij.  Energy e_i = 1/2 sum_j U (minus U(rc_i) per pair if shifted),     */
/* virial W = 1/2 sum_i sum_j r_ij . F_ij.                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int ntypes;
  double eps[16];   /* per type pair a*ntypes+b */
  double sig2[16];
} ljtab_t;

static void lj_table(int ntypes, const double* eps, const double* sigma, ljtab_t* t) {
  t->ntypes = ntypes;
  for (int a = 0; a < ntypes; ++a)
    for (int b = 0; b < ntypes; ++b) {
      double e = sqrt(eps[a] * eps[b]);
      double s = 0.5 * (sigma[a] + sigma[b]);
      t->eps[a * ntypes + b] = e;
      t->sig2[a * ntypes + b] = s * s;
    }
}

static double min_image(double d, double L) {
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}

static void lj_pair(double r2, double eps, double sig2, double* fscal, double* u) {
  double s2 = sig2 / r2;
  double s6 = s2 * s2 * s2;
  *fscal = 24.0 * eps * (2.0 * s6 * s6 - s6) / r2;
  *u = 4.0 * eps * (s6 * s6 - s6);
}

static void accumulate_pair(const double* pi, const double* pj, int ti, int tj, double rci,
                            const double* L, const ljtab_t* tab, int shift, double* f, double* e,
                            double* w, int64_t* np) {
  double dx = min_image(pi[0] - pj[0], L[0]);
  double dy = min_image(pi[1] - pj[1], L[1]);
  double dz = min_image(pi[2] - pj[2], L[2]);
  double r2 = dx * dx + dy * dy + dz * dz;
  if (!(r2 < rci * rci)) return;
  int pt = ti * tab->ntypes + tj;
  double fs, u;
  lj_pair(r2, tab->eps[pt], tab->sig2[pt], &fs, &u);
  if (shift) {
    double fc, uc;
    lj_pair(rci * rci, tab->eps[pt], tab->sig2[pt], &fc, &uc);
    u -= uc;
  }
  f[0] += fs * dx;
  f[1] += fs * dy;
  f[2] += fs * dz;
  *e += 0.5 * u;
  *w += 0.5 * fs * r2;
  *np += 1;
}

/* O(N^2) reference: every ordered pair (i, j != i).  out[0] = E, out[1] = W;
 * npairs = number of accepted ordered pairs. */
void orc_forces_brute(int64_t n, const double* pos, const int32_t* type, const double* rc,
                      const double* L, int ntypes, const double* eps, const double* sigma, int shift,
                      double* F, double* e, double* out, int64_t* npairs) {
  ljtab_t tab;
  lj_table(ntypes, eps, sigma, &tab);
  double E = 0.0, W = 0.0;
  int64_t np = 0;
  for (int64_t i = 0; i < n; ++i) {
    double f[3] = {0, 0, 0}, ei = 0.0, wi = 0.0;
    int ti = type ? type[i] : 0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      accumulate_pair(pos + 3 * i, pos + 3 * j, ti, type ? type[j] : 0, rc[i], L, &tab, shift, f, &ei, &wi, &np);
    }
    F[3 * i] = f[0];
    F[3 * i + 1] = f[1];
    F[3 * i + 2] = f[2];
    if (e) e[i] = ei;
    E += ei;
    W += wi;
  }
  out[0] = E;
  out[1] = W;
  if (npairs) *npairs = np;
}

/* Forces of one particle i over the bins around it (shared by the two
 * cell-list entry points below). */
static void cells_one(int64_t i, const double* pos, const int32_t* type, const double* rc, const double* L,
                      const double* l, const int64_t* nc, const ljtab_t* tab, int shift, const int32_t* cell,
                      const int32_t* start, const int32_t* perm, double* f, double* ei, double* wi, int64_t* np) {
  int ti = type ? type[i] : 0;
  int64_t c = cell[i];
  int64_t cc[3] = {c % nc[0], (c / nc[0]) % nc[1], c / (nc[0] * nc[1])};
  int64_t lo[3], cnt[3];
  for (int d = 0; d < 3; ++d) {
    int64_t H = (int64_t)ceil(rc[i] / l[d]);
    if (2 * H + 1 >= nc[d]) {
      lo[d] = 0;
      cnt[d] = nc[d];
    } else {
      lo[d] = cc[d] - H;
      cnt[d] = 2 * H + 1;
    }
  }
  for (int64_t a = 0; a < cnt[2]; ++a) {
    int64_t jz = wrap(lo[2] + a, nc[2]);
    for (int64_t b = 0; b < cnt[1]; ++b) {
      int64_t jy = wrap(lo[1] + b, nc[1]);
      for (int64_t k = 0; k < cnt[0]; ++k) {
        int64_t jx = wrap(lo[0] + k, nc[0]);
        int64_t jc = jx + nc[0] * (jy + nc[1] * jz);
        for (int32_t s = start[jc]; s < start[jc + 1]; ++s) {
          int64_t j = perm[s];
          if (j == i) continue;
          accumulate_pair(pos + 3 * i, pos + 3 * j, ti, type ? type[j] : 0, rc[i], L, tab, shift, f, ei, wi, np);
        }
      }
    }
  }
}

/* Forces, energies, virials and accepted-pair counts of the m particles
 * idx[0..m) only (the full system is binned); used to check large systems on
 * a sample of particles. */
void orc_forces_subset(int64_t n, const double* pos, const int32_t* type, const double* rc, const double* L,
                       const double* l, const int64_t* nc, int ntypes, const double* eps, const double* sigma,
                       int shift, int64_t m, const int64_t* idx, int nthreads, double* F, double* e, double* w,
                       int64_t* np) {
  ljtab_t tab;
  lj_table(ntypes, eps, sigma, &tab);
  int64_t ncell = nc[0] * nc[1] * nc[2];
  int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* count = (int32_t*)malloc(sizeof(int32_t) * (size_t)ncell);
  int32_t* start = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  orc_bin(n, pos, l, nc, cell, count, start, perm);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 20)
#endif
  for (int64_t k = 0; k < m; ++k) {
    double f[3] = {0, 0, 0}, ei = 0.0, wi = 0.0;
    int64_t p = 0;
    cells_one(idx[k], pos, type, rc, L, l, nc, &tab, shift, cell, start, perm, f, &ei, &wi, &p);
    F[3 * k] = f[0];
    F[3 * k + 1] = f[1];
    F[3 * k + 2] = f[2];
    e[k] = ei;
    w[k] = wi;
    np[k] = p;
  }
  free(cell);
  free(count);
  free(start);
  free(perm);
}

/* Cell-list form (Algorithm 2.2's bins and Algorithm 2.3's loop fused): bin
 * with edge l, then for every i visit all bins within ceil(rc_i / l) bins in
 * each direction (each bin once, even if the stencil wraps past the box) and
 * apply the same pair rule.  The i-loop is shared among threads with the
 * paper's dynamic schedule of 20 particles per task (Section 2.4). */
void orc_forces_cells(int64_t n, const double* pos, const int32_t* type, const double* rc,
                      const double* L, const double* l, const int64_t* nc, int ntypes,
                      const double* eps, const double* sigma, int shift, int nthreads, double* F,
                      double* e, double* out, int64_t* npairs) {
  ljtab_t tab;
  lj_table(ntypes, eps, sigma, &tab);
  int64_t ncell = nc[0] * nc[1] * nc[2];
  int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* count = (int32_t*)malloc(sizeof(int32_t) * (size_t)ncell);
  int32_t* start = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  double* wl = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* el = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int64_t* pl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  orc_bin(n, pos, l, nc, cell, count, start, perm);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 20)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double f[3] = {0, 0, 0}, ei = 0.0, wi = 0.0;
    int64_t np = 0;
    cells_one(i, pos, type, rc, L, l, nc, &tab, shift, cell, start, perm, f, &ei, &wi, &np);
    F[3 * i] = f[0];
    F[3 * i + 1] = f[1];
    F[3 * i + 2] = f[2];
    el[i] = ei;
    wl[i] = wi;
    pl[i] = np;
  }
  double E = 0.0, W = 0.0;
  int64_t np = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (e) e[i] = el[i];
    E += el[i];
    W += wl[i];
    np += pl[i];
  }
  out[0] = E;
  out[1] = W;
  if (npairs) *npairs = np;
  free(cell);
  free(count);
  free(start);
  free(perm);
  free(wl);
  free(el);
  free(pl);
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the force/energy map (extension for differentiation).          */
/* For a scalar loss L(F, E) with upstream A_i = dL/dF_i and dLdE = dL/dE,    */
/* cutoffs held fixed:                                                       */
/*   dL/dr_k = sum_{j in N(k)} [ J(r_kj) A_k - dLdE/2 phi_kj ]               */
/*           + sum_{j : k in N(j)} [ -J(r_kj) A_j - dLdE/2 phi_kj ]          */
/* with N(i) = {j != i : |r_ij| < rc_i}, phi_ij = g(r) r_ij the force on i   */
/* from j, g(r) = 24 eps [2 (s/r)^12 - (s/r)^6] / r^2 and the (symmetric)    */
/* Jacobian J(r) = d phi / d r_i = g I + (g'(r) / r) r r^T,                  */
/* g'(r) / r = 24 eps [-28 (s/r)^12 + 8 (s/r)^6] / r^4.                       */
/* Per type pair p = (a, b) of a forward pair (i, j in N(i)):                */
/*   dL/deps_p   += A_i . phi_ij / eps_p + dLdE/2 (U - Ushift) / eps_p        */
/*   dL/dsigma_p += A_i . dphi/dsigma + dLdE/2 d(U - Ushift)/dsigma           */
/* with dg/dsigma = (24 eps / sigma) [24 (s/r)^12 - 6 (s/r)^6] / r^2 and      */
/* dU/dsigma = (4 eps / sigma) [12 (s/r)^12 - 6 (s/r)^6] (Ushift = U(rc_i)).  */
/* O(N^2) over all ordered pairs.                                            */
/* ------------------------------------------------------------------------ */
static void lj_terms(double r2, double eps, double sig2, double* g, double* gpr, double* u) {
  double s2 = sig2 / r2;
  double s6 = s2 * s2 * s2, s12 = s6 * s6;
  *g = 24.0 * eps * (2.0 * s12 - s6) / r2;
  *gpr = 24.0 * eps * (-28.0 * s12 + 8.0 * s6) / (r2 * r2);
  *u = 4.0 * eps * (s12 - s6);
}

void orc_adjoint_brute(int64_t n, const double* pos, const int32_t* type, const double* rc, const double* L,
                       int ntypes, const double* eps, const double* sigma, int shift, const double* A,
                       double dLdE, double* G, double* deps_pair, double* dsig_pair) {
  ljtab_t tab;
  lj_table(ntypes, eps, sigma, &tab);
  for (int p = 0; p < ntypes * ntypes; ++p) deps_pair[p] = dsig_pair[p] = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    double gk[3] = {0, 0, 0};
    int tk = type ? type[k] : 0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == k) continue;
      int tj = type ? type[j] : 0;
      double r[3] = {min_image(pos[3 * k] - pos[3 * j], L[0]), min_image(pos[3 * k + 1] - pos[3 * j + 1], L[1]),
                     min_image(pos[3 * k + 2] - pos[3 * j + 2], L[2])};
      double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
      int p = tk * ntypes + tj;
      double g, gpr, u;
      lj_terms(r2, tab.eps[p], tab.sig2[p], &g, &gpr, &u);
      int fwd = r2 < rc[k] * rc[k];  /* j in N(k)  */
      int rev = r2 < rc[j] * rc[j];  /* k in N(j)  */
      if (fwd) {
        const double* a = A + 3 * k;
        double ra = r[0] * a[0] + r[1] * a[1] + r[2] * a[2];
        for (int d = 0; d < 3; ++d) gk[d] += g * a[d] + gpr * ra * r[d] - 0.5 * dLdE * g * r[d];
        /* parameter gradients of the forward pair (k, j) */
        double e = tab.eps[p], sg = sqrt(tab.sig2[p]);
        double s2 = tab.sig2[p] / r2, s6 = s2 * s2 * s2, s12 = s6 * s6;
        double dg_dsig = 24.0 * e / sg * (24.0 * s12 - 6.0 * s6) / r2;
        double du_dsig = 4.0 * e / sg * (12.0 * s12 - 6.0 * s6);
        double uc = 0.0, duc_dsig = 0.0;
        if (shift) {
          double c2 = tab.sig2[p] / (rc[k] * rc[k]), c6 = c2 * c2 * c2, c12 = c6 * c6;
          uc = 4.0 * e * (c12 - c6);
          duc_dsig = 4.0 * e / sg * (12.0 * c12 - 6.0 * c6);
        }
        deps_pair[p] += (g * ra) / e + 0.5 * dLdE * (u - uc) / e;
        dsig_pair[p] += dg_dsig * ra + 0.5 * dLdE * (du_dsig - duc_dsig);
      }
      if (rev) {
        const double* a = A + 3 * j;
        double ra = r[0] * a[0] + r[1] * a[1] + r[2] * a[2];
        for (int d = 0; d < 3; ++d) gk[d] += -(g * a[d] + gpr * ra * r[d]) - 0.5 * dLdE * g * r[d];
      }
    }
    G[3 * k] = gk[0];
    G[3 * k + 1] = gk[1];
    G[3 * k + 2] = gk[2];
  }
}

/* ------------------------------------------------------------------------ */
/* Velocity Verlet (Section 2, box 5 of Fig. 3), unit masses.                */
/* ------------------------------------------------------------------------ */
void orc_kick(int64_t n, double* vel, const double* F, double half_dt) {
  for (int64_t k = 0; k < 3 * n; ++k) vel[k] += half_dt * F[k];
}

/* Drift and wrap into [0, L). */
void orc_drift(int64_t n, double* pos, const double* vel, double dt, const double* L) {
  for (int64_t i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      double x = pos[3 * i + d] + dt * vel[3 * i + d];
      if (x >= L[d]) x -= L[d];
      if (x < 0.0) x += L[d];
      if (x >= L[d]) x = 0.0;
      pos[3 * i + d] = x;
    }
}

double orc_kinetic(int64_t n, const double* vel) {
  double k = 0.0;
  for (int64_t i = 0; i < 3 * n; ++i) k += 0.5 * vel[i] * vel[i];
  return k;
}
