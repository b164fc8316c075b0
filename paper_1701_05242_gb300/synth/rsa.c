/*
 * Seeded synthetic liquid/vapor slab generator (random sequential addition).
 *
 * This file generates INPUTS only: particle positions drawn uniformly inside a
 * liquid region (a slab between two surfaces z_lo(x,y) <= z < z_hi(x,y)) and a
 * vapor region (the rest of the periodic box), rejecting any proposal that
 * lies closer than d_min to an already placed particle (periodic minimum
 * image).  It contains none of the dynamic-cutoff method's arithmetic and is
 * shared by the FP64 oracle and the CUDA path, which both consume the arrays it
 * writes.
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based
 * generator: value k of stream s is mix(s * GOLDEN + k * GOLDEN'), so the
 * output is identical on every platform (integer arithmetic only; doubles are
 * formed from the top 53 bits).
 *
 * Surfaces: z_s(x,y) = z0_s + sum_m A_m cos(2*pi*(kx_m x/Lx + ky_m y/Ly) + phi_m),
 * with the mode table supplied by the caller (empty table => planar slab).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

typedef struct {
  uint64_t base;
  uint64_t k;
} rng_t;

static double rng_u01(rng_t* r) {
  uint64_t x = sm64_mix(r->base + (r->k++) * 0x9e3779b97f4a7c15ULL);
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

typedef struct {
  int nm;
  const double *kx, *ky, *amp, *phase;
  double z0;
} surface_t;

static double surface_z(const surface_t* s, double x, double y, double Lx, double Ly) {
  double z = s->z0;
  const double twopi = 6.283185307179586476925286766559;
  for (int m = 0; m < s->nm; ++m)
    z += s->amp[m] * cos(twopi * (s->kx[m] * x / Lx + s->ky[m] * y / Ly) + s->phase[m]);
  return z;
}

/* Periodic proximity grid: head[cell] -> particle, next[particle] -> particle. */
typedef struct {
  int nx, ny, nz;
  double cx, cy, cz; /* cell edges (>= d_min) */
  int32_t* head;
  int32_t* next;
} grid_t;

static int to_float_coord(double v, double L, float* out) {
  float f = (float)v;
  if (!(f >= 0.0f)) f = 0.0f;
  if (f >= (float)L) f = 0.0f; /* wraps L onto 0 */
  *out = f;
  return 0;
}

static int too_close(const grid_t* g, const float* pos, double x, double y, double z,
                     double Lx, double Ly, double Lz, double dmin2) {
  int ix = (int)floor(x / g->cx), iy = (int)floor(y / g->cy), iz = (int)floor(z / g->cz);
  if (ix >= g->nx) ix = g->nx - 1;
  if (iy >= g->ny) iy = g->ny - 1;
  if (iz >= g->nz) iz = g->nz - 1;
  int rx = g->nx < 3 ? g->nx : 3, ry = g->ny < 3 ? g->ny : 3, rz = g->nz < 3 ? g->nz : 3;
  for (int a = 0; a < rz; ++a) {
    int jz = iz - 1 + a;
    jz = jz < 0 ? jz + g->nz : (jz >= g->nz ? jz - g->nz : jz);
    for (int b = 0; b < ry; ++b) {
      int jy = iy - 1 + b;
      jy = jy < 0 ? jy + g->ny : (jy >= g->ny ? jy - g->ny : jy);
      for (int c = 0; c < rx; ++c) {
        int jx = ix - 1 + c;
        jx = jx < 0 ? jx + g->nx : (jx >= g->nx ? jx - g->nx : jx);
        for (int32_t p = g->head[(int64_t)jx + (int64_t)g->nx * (jy + (int64_t)g->ny * jz)]; p >= 0;
             p = g->next[p]) {
          double dx = x - pos[3 * (int64_t)p], dy = y - pos[3 * (int64_t)p + 1],
                 dz = z - pos[3 * (int64_t)p + 2];
          if (dx > 0.5 * Lx) dx -= Lx; else if (dx < -0.5 * Lx) dx += Lx;
          if (dy > 0.5 * Ly) dy -= Ly; else if (dy < -0.5 * Ly) dy += Ly;
          if (dz > 0.5 * Lz) dz -= Lz; else if (dz < -0.5 * Lz) dz += Lz;
          if (dx * dx + dy * dy + dz * dz < dmin2) return 1;
        }
      }
    }
  }
  return 0;
}

/*
 * Fill the box slab by slab along z (nslab equal slabs, processed in order).
 * Slab k receives exactly q_liq[k] liquid and q_vap[k] vapor particles:
 * proposals are uniform in the slab, classified by the surfaces, discarded if
 * their phase is already full, and rejected if closer than d_min to any
 * particle already placed (in this or an earlier slab, periodic).  Filling
 * slab by slab keeps the working set local, so large systems generate fast.
 * Writes float32 xyz into pos[3*n] (liquid first, then vapor, each in slab
 * order) and returns 0; -1 if max_tries_per_particle consecutive proposals
 * failed (density too high for d_min), -2 on allocation failure.
 */
/* Liquid region: a slab between two surfaces (cyl_r <= 0), or the cylinder
 * (y - cyl_y)^2 + (z - cyl_z)^2 < cyl_r^2 along x (cyl_r > 0). */
typedef struct {
  surface_t lo, hi;
  double reach_lo, reach_hi;
  double cyl_r, cyl_y, cyl_z;
  double Lx, Ly;
} region_t;

static int in_liquid(const region_t* q, double x, double y, double z) {
  if (q->cyl_r > 0.0) {
    double dy = y - q->cyl_y, dz = z - q->cyl_z;
    return dy * dy + dz * dz < q->cyl_r * q->cyl_r;
  }
  if (z >= q->lo.z0 + q->reach_lo && z < q->hi.z0 - q->reach_hi) return 1;
  if (z < q->lo.z0 - q->reach_lo || z >= q->hi.z0 + q->reach_hi) return 0;
  double zl = surface_z(&q->lo, x, y, q->Lx, q->Ly), zh = surface_z(&q->hi, x, y, q->Lx, q->Ly);
  return z >= zl && z < zh;
}

static int rsa_fill(double Lx, double Ly, double Lz, int nslab, const int64_t* q_liq, const int64_t* q_vap,
                    double d_min, uint64_t seed, const region_t* region, int64_t max_tries_per_particle,
                    float* pos);

int synth_rsa_slab(double Lx, double Ly, double Lz, int nslab, const int64_t* q_liq,
                   const int64_t* q_vap, double d_min, uint64_t seed, int nm_lo,
                   const double* kx_lo, const double* ky_lo, const double* amp_lo,
                   const double* ph_lo, double z0_lo, int nm_hi, const double* kx_hi,
                   const double* ky_hi, const double* amp_hi, const double* ph_hi, double z0_hi,
                   int64_t max_tries_per_particle, float* pos) {
  region_t q;
  q.lo = (surface_t){nm_lo, kx_lo, ky_lo, amp_lo, ph_lo, z0_lo};
  q.hi = (surface_t){nm_hi, kx_hi, ky_hi, amp_hi, ph_hi, z0_hi};
  q.reach_lo = 1e-12;
  q.reach_hi = 1e-12;
  for (int m = 0; m < nm_lo; ++m) q.reach_lo += fabs(amp_lo[m]);
  for (int m = 0; m < nm_hi; ++m) q.reach_hi += fabs(amp_hi[m]);
  q.cyl_r = 0.0;
  q.cyl_y = q.cyl_z = 0.0;
  q.Lx = Lx;
  q.Ly = Ly;
  return rsa_fill(Lx, Ly, Lz, nslab, q_liq, q_vap, d_min, seed, &q, max_tries_per_particle, pos);
}

/* The same fill with a liquid cylinder of radius r along x, axis at (y0, z0). */
int synth_rsa_cylinder(double Lx, double Ly, double Lz, int nslab, const int64_t* q_liq, const int64_t* q_vap,
                       double d_min, uint64_t seed, double r, double y0, double z0,
                       int64_t max_tries_per_particle, float* pos) {
  region_t q;
  q.lo = (surface_t){0, 0, 0, 0, 0, 0.0};
  q.hi = q.lo;
  q.reach_lo = q.reach_hi = 0.0;
  q.cyl_r = r;
  q.cyl_y = y0;
  q.cyl_z = z0;
  q.Lx = Lx;
  q.Ly = Ly;
  return rsa_fill(Lx, Ly, Lz, nslab, q_liq, q_vap, d_min, seed, &q, max_tries_per_particle, pos);
}

static int rsa_fill(double Lx, double Ly, double Lz, int nslab, const int64_t* q_liq, const int64_t* q_vap,
                    double d_min, uint64_t seed, const region_t* region, int64_t max_tries_per_particle,
                    float* pos) {
  grid_t g;
  g.nx = (int)floor(Lx / d_min);
  g.ny = (int)floor(Ly / d_min);
  g.nz = (int)floor(Lz / d_min);
  if (g.nx < 1) g.nx = 1;
  if (g.ny < 1) g.ny = 1;
  if (g.nz < 1) g.nz = 1;
  g.cx = Lx / g.nx;
  g.cy = Ly / g.ny;
  g.cz = Lz / g.nz;
  int64_t ncell = (int64_t)g.nx * g.ny * g.nz;
  int64_t n_liq = 0, n = 0;
  for (int k = 0; k < nslab; ++k) {
    n_liq += q_liq[k];
    n += q_liq[k] + q_vap[k];
  }
  g.head = (int32_t*)malloc(sizeof(int32_t) * (size_t)ncell);
  g.next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!g.head || !g.next) {
    free(g.head);
    free(g.next);
    return -2;
  }
  for (int64_t c = 0; c < ncell; ++c) g.head[c] = -1;
  rng_t r = {sm64_mix(seed ^ 0x5851f42d4c957f2dULL), 0};
  double dmin2 = d_min * d_min;
  int64_t next_liq = 0, next_vap = n_liq; /* output slots */
  for (int k = 0; k < nslab; ++k) {
    double za = Lz * k / nslab, zb = Lz * (k + 1) / nslab;
    int64_t left_liq = q_liq[k], left_vap = q_vap[k], tries = 0;
    while (left_liq > 0 || left_vap > 0) {
      if (++tries > max_tries_per_particle) {
        free(g.head);
        free(g.next);
        return -1;
      }
      double x = rng_u01(&r) * Lx, y = rng_u01(&r) * Ly;
      double z = za + rng_u01(&r) * (zb - za);
      float fx, fy, fz;
      to_float_coord(x, Lx, &fx);
      to_float_coord(y, Ly, &fy);
      to_float_coord(z, Lz, &fz);
      int inside = in_liquid(region, fx, fy, fz);
      if (inside ? left_liq == 0 : left_vap == 0) continue;
      if (too_close(&g, pos, fx, fy, fz, Lx, Ly, Lz, dmin2)) continue;
      int64_t slot = inside ? next_liq++ : next_vap++;
      if (inside)
        --left_liq;
      else
        --left_vap;
      pos[3 * slot] = fx;
      pos[3 * slot + 1] = fy;
      pos[3 * slot + 2] = fz;
      int ix = (int)floor(fx / g.cx), iy = (int)floor(fy / g.cy), iz = (int)floor(fz / g.cz);
      if (ix >= g.nx) ix = g.nx - 1;
      if (iy >= g.ny) iy = g.ny - 1;
      if (iz >= g.nz) iz = g.nz - 1;
      int64_t c = (int64_t)ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz);
      g.next[slot] = g.head[c];
      g.head[c] = (int32_t)slot;
      tries = 0;
    }
  }
  free(g.head);
  free(g.next);
  return 0;
}

/* Counter-based uniform draws for callers that need them: out[i] = U[0,1) of
 * stream `seed`, counter `offset + i`. */
void synth_uniform(uint64_t seed, uint64_t offset, int64_t n, double* out) {
  rng_t r = {sm64_mix(seed ^ 0x5851f42d4c957f2dULL), offset};
  for (int64_t i = 0; i < n; ++i) out[i] = rng_u01(&r);
}
