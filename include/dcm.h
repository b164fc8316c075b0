/*
 * dcm.h - C ABI of the GB300 (sm_103a) implementation of the per-timestep hot
 * path of the Dynamic Cutoff Method (DCM) of Springer, Ismail and Bientinesi,
 * "A Scalable, Linear-Time Dynamic Cutoff Algorithm for Molecular Dynamics".
 *
 * The path of one timestep (Fig. 3 of the paper, boxes 1-5):
 *   dcm_bin               particles -> cells (Sections 2.1 and 2.3)
 *   dcm_box_counts        particles -> particle count per density box (Sec. 2.1)
 *   dcm_detect_interface  counts -> gray-scale volume -> segmented volume S
 *                         (Eq. 4) -> interface boxes (Section 2.1)
 *   dcm_distance          S, interface -> box-interface distances D by
 *                         cutoff-based fast sweeping (Section 2.2, Alg. 2.1)
 *   dcm_cutoffs           D -> particle-interface distance (trilinear) ->
 *                         per-particle cutoff rc_i (Section 2.2)
 *   dcm_forces            i-centric Lennard-Jones force and energy with
 *                         per-particle cutoffs, no Newton's third law
 *                         (Section 2.4, Algorithms 2.2 and 2.3)
 *   dcm_step              velocity Verlet around all of the above (Section 2)
 *
 * Conventions shared by every call
 * --------------------------------
 * - All array arguments are DEVICE pointers owned by the caller, unless a
 *   parameter says "host".  The library never frees them.  The library owns
 *   only the scratch inside a dcm_ctx (allocated once by dcm_create).
 * - Every call is asynchronous on the given stream unless documented
 *   otherwise; a call returns after enqueuing its kernels.  Calls on one
 *   context must not overlap in time on different streams (they share the
 *   context's scratch).
 * - Every call returns DCM_OK (0) or a DCM_ERR_* code; dcm_last_error() gives
 *   a message for the last failing call on that context.  Kernels never trap:
 *   device-side failures (capacity, non-convergence) are written to a device
 *   status word that dcm_status() reads.
 * - Precision forms (dcm_params.precision):
 *     DCM_PREC_MIXED: positions/velocities/forces are float4, cutoffs and
 *       distances float; pair arithmetic in FP32, per-particle sums as
 *       dcm_params.accumulation says (compensated by default),
 *       energy/virial/kinetic totals reduced in FP64.
 *     DCM_PREC_FP64:  the same arrays as double4 / double; all arithmetic FP64.
 *   "real4" below means float4 or double4 accordingly, "real" float or double.
 * - Positions are real4 {x, y, z, w}: w holds the particle type as a number
 *   (0, 1, ...; 0 for one-type systems).  Coordinates must lie in [0, L);
 *   finite values outside are clamped into the boundary cells by the binning
 *   and take part in no pair farther than their cutoff (a NaN or infinite
 *   coordinate turns the forces of its cell neighbours into NaN).  No value
 *   makes a kernel read or write outside its arrays.
 * - Forces are real4 {fx, fy, fz, e_i}: e_i is the particle's energy (half of
 *   every accepted pair's U).
 * - Cell and box indices are linear: c = cx + nx * (cy + ny * cz).
 */
#ifndef DCM_H
#define DCM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque CUDA stream (same object as cudaStream_t; NULL = legacy default stream). */
typedef struct CUstream_st* dcm_stream_t;

enum dcm_status_code {
  DCM_OK = 0,
  DCM_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad parameter */
  DCM_ERR_BOX = 2,           /* box not a multiple of l or h, rc_max > L/2, bad edge */
  DCM_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed */
  DCM_ERR_NOT_CONVERGED = 4, /* fast sweeping did not converge within iter_max */
  DCM_ERR_CAPACITY = 5,      /* n > n_max, or a density value range beyond the histogram */
  DCM_ERR_NOMEM = 6,         /* scratch allocation failed in dcm_create */
  DCM_ERR_TIMEOUT = 7        /* a device-side wait ran past its budget (a grid barrier, the cell-count scan) */
};

/* Cell-list force kernels (both walk the same culled cell rows and accept the
 * same pairs; they differ in how the pair arithmetic is issued).  The packed
 * kernel serves FP32 runs (DCM_PREC_MIXED) of one or two types; otherwise
 * kernel 1 runs.  Values 2, 4 and 5 are not used (invalid). */
enum {
  DCM_FORCE_AUTO = 0,        /* kernel 3 where it applies, else kernel 1 */
  DCM_FORCE_THREAD = 1,      /* one thread per particle i, one candidate per instruction */
  DCM_FORCE_PACKED = 3       /* one thread per particle i, two candidates per FP32x2 instruction */
};

/* Per-particle accumulation of the mixed precision form (dcm_params.
 * accumulation): how the FP32 pair terms of particle i (its force, energy and
 * virial) are summed.  Totals E and W are always reduced in FP64.  A "row
 * segment" is one contiguous run of candidates j of the cell-row walk (at
 * most a row of cells: about ten candidates at rc = 3).
 *   DCM_ACC_FP32       plain FP32 running sums
 *   DCM_ACC_ROW_FP64   FP32 sum per row segment, segment sums added in FP64
 *   DCM_ACC_ROW_KAHAN  FP32 sum per row segment, segment sums added with
 *                      Kahan compensation in FP32
 *   DCM_ACC_PAIR_KAHAN every pair term added with Kahan compensation (FP32)
 *   DCM_ACC_PAIR_FP64  every pair term added in FP64
 *   DCM_ACC_PLANE_FP64 FP32 sum per z-plane of the stencil (its rows: up to
 *                      five at rc = 3), plane sums added in FP64
 *   DCM_ACC_PLANE_KAHAN the same, plane sums Kahan-compensated in FP32
 *   DCM_ACC_AUTO (0)   DCM_ACC_PLANE_KAHAN, the cheapest of the compensated
 *                      forms at the accuracy of the FP64 ones (measured)
 * The pair forms run on the packed kernel; the scalar FP32 kernel (three or
 * four types) runs their row form instead.  The FP64 precision form ignores
 * this field (everything is FP64). */
enum dcm_accumulation {
  DCM_ACC_AUTO = 0,
  DCM_ACC_FP32 = 1,
  DCM_ACC_ROW_FP64 = 2,
  DCM_ACC_ROW_KAHAN = 3,
  DCM_ACC_PAIR_KAHAN = 4,
  DCM_ACC_PAIR_FP64 = 5,
  DCM_ACC_PLANE_FP64 = 6,
  DCM_ACC_PLANE_KAHAN = 7
};

enum dcm_precision { DCM_PREC_FP64 = 0, DCM_PREC_MIXED = 1 };

/* Parameters of one system.  dcm_params_default() fills the defaults used for
 * the liquid/vapor slabs (reduced LJ units). */
typedef struct dcm_params {
  double box[3];          /* periodic box lengths Lx, Ly, Lz */
  double h;               /* density-box edge (Section 2.1, footnote 2); L/h integer. Default 1.5 */
  double l;               /* force-cell edge (Section 2.3: l <= rc_min); L/l integer. Default 1.5 */
  double rc_min;          /* smallest cutoff (Section 2.2). Default 3.0 */
  double rc_max;          /* largest cutoff, at the interface and in vapor. Default 6.0 */
  double ramp;            /* distance over which rc falls from rc_max to rc_min; <= 0 -> rc_max - rc_min */
  double r_grid;          /* CFSM threshold r_c^grid (Alg. 2.1); <= 0 -> ramp + 2 h */
  int32_t smooth_w;       /* gray-scale box-sum half width (boxes). Default 2 */
  int32_t threshold;      /* < 0: 2-means threshold; >= 0: fixed threshold T on the box sums */
  int32_t iter_max;       /* CFSM iteration cap (Alg. 2.1). Default 1000 */
  int32_t ntypes;         /* 1..4 particle types */
  double eps[4];          /* per-type LJ epsilon (Lorentz-Berthelot: sqrt(eps_a eps_b)) */
  double sigma[4];        /* per-type LJ sigma   (Lorentz-Berthelot: (sigma_a + sigma_b)/2) */
  int32_t shift_energy;   /* 1: pair energy U(r) - U(rc_i); forces unchanged. Default 0 */
  int32_t precision;      /* DCM_PREC_MIXED (default) or DCM_PREC_FP64 */
  int32_t recompute_every;/* K: interface, distances and cutoffs every K steps. Default 10 */
  int32_t force_kernel;   /* cell-list force kernel (DCM_FORCE_*); DCM_FORCE_AUTO (0) by default */
  int64_t n_max;          /* largest particle count any call on this context will pass */
  double skin;            /* > 0: dcm_step keeps Verlet neighbour lists of radius rc_i + skin
                             (Algorithm 2.2) and rebuilds them only when a particle has moved
                             more than skin / 2 since the last build or the cutoffs are
                             recomputed; 0 (default): forces straight from the cell lists */
  int32_t min_component;  /* > 0: remove connected components of S (6-connected, periodic, either
                             phase) of fewer boxes before the interface is taken (Section 2.1's
                             bubble filter); 0 (default): off.  Single-system contexts only */
  int32_t accumulation;   /* DCM_ACC_*: per-particle sums of the mixed form. Default DCM_ACC_AUTO */
  double lx;              /* force-cell edge along x, the direction in which a row of cells is one
                             contiguous run of sorted particles; L_x / lx integer, short mantissa
                             (for a batch: every replica's L_x).  0 (default): l.  Finer cells
                             along the rows narrow each row's window without adding rows */
  int32_t newton3;        /* 1 (needs skin > 0): half Verlet lists, each pair kept once by the
                             particle with the larger cutoff (lower index on a tie) and evaluated
                             once: the force goes to that particle if |r| < its cutoff and, with
                             the opposite sign, to the other if |r| < the other's cutoff (Newton's
                             third law where both cutoffs reach, Section 4.2; i-centric where one
                             does).  Results are summed with atomics (order not reproducible).
                             0 (default): full i-centric lists */
  int32_t segmentation;   /* 0 (default): S = threshold of the box sums (2-means or fixed);
                             1: then refined by the regularised two-phase Mumford-Shah
                             segmentation of the unsmoothed box counts (Section 2.1): phase
                             values c0, c1 = the phase means, s minimising
                             sum (g - c_s)^2 + ms_nu x (faces between the phases), by a
                             primal-dual iteration on the convex relaxation thresholded at 1/2.
                             Single-system contexts only */
  int32_t ms_inner;       /* primal-dual iterations per outer iteration (1..100000). Default 200 */
  int32_t ms_outer;       /* outer iterations (phase values, then s) at most (1..64). Default 4 */
  int32_t reserved4;
  double ms_nu;           /* weight of the length term, in (box count)^2 (>= 0). Default 4 */
} dcm_params;

typedef struct dcm_ctx dcm_ctx;

/* Particle state for dcm_step.  Each array has two buffers; the step reads
 * buffer `cur`, writes the cell-sorted particles into buffer 1-cur and flips
 * `cur`.  pos/vel/force are real4[n]; rc is real[n] (the particle's cutoff,
 * which travels with it between recomputations); id is int32[n] (any payload
 * that travels with the particle, e.g. its original index).  thermo is
 * double[4] on the device: {E, W, KE, accepted pairs} after the last step.
 * t counts timesteps since dcm_step_init (recomputation when t % K == 0). */
typedef struct dcm_state {
  void* pos[2];
  void* vel[2];
  void* rc[2];
  int32_t* id[2];
  void* force;
  double* thermo;
  int32_t cur;
  int32_t reserved;
  int64_t t;
} dcm_state;

/* ---- host-only helpers (no GPU needed) -------------------------------- */

/* Fill *p with defaults (box left at 0). Returns DCM_OK or DCM_ERR_INVALID_ARG. */
int dcm_params_default(dcm_params* p);

/* Check *p without touching the GPU.  Rules: box > 0; h and l have at most 8
 * significant bits (so k*l is exact in FP32) and divide every box length
 * into fewer than 65536 cells, fewer than 2^31 cells (and boxes) in all;
 * 0 < rc_min <= rc_max <= min(L)/2 (so at most one periodic image of a
 * particle lies within any cutoff); 1 <= ntypes <= 4; eps, sigma > 0;
 * smooth_w >= 0; 1 <= iter_max <= 100000; recompute_every >= 1;
 * force_kernel one of DCM_FORCE_*; min_component >= 0; 0 <= n_max < 2^31;
 * skin >= 0 with rc_max + skin <= min(L)/2 and n_max < 2^26 when skin > 0.
 * On failure writes a message to msg (if msg_len > 0) and returns
 * DCM_ERR_BOX, DCM_ERR_INVALID_ARG or DCM_ERR_CAPACITY. */
int dcm_validate_params(const dcm_params* p, char* msg, int32_t msg_len);

/* Grid shapes for a parameter set: cells3 = force cells per dimension (L/l),
 * boxes3 = density boxes per dimension (L/h).  Host-only. */
int dcm_grid_dims(const dcm_params* p, int64_t* cells3, int64_t* boxes3);

/* Bytes of device scratch dcm_create allocates for *p (host-only). */
int dcm_scratch_bytes(const dcm_params* p, int64_t* bytes);

/* Library version string (host-only). */
const char* dcm_version(void);

/* ---- context ----------------------------------------------------------- */

/* Validate *p, then allocate the context and its device scratch on the
 * current CUDA device (synchronous).  *out receives the context. */
int dcm_create(const dcm_params* p, dcm_ctx** out);

/* Free the context and its scratch (synchronous).  NULL is a no-op. */
void dcm_destroy(dcm_ctx* ctx);

/* Message of the last failing call on ctx ("" if none). */
const char* dcm_last_error(const dcm_ctx* ctx);

/* Synchronise `stream`, read and clear the device status word of ctx.
 * Returns DCM_OK or the first device-side error recorded since the last call
 * (DCM_ERR_NOT_CONVERGED, DCM_ERR_CAPACITY). */
int dcm_status(dcm_ctx* ctx, dcm_stream_t stream);

/* Self-test of the failure path of the cell-count scan (the single-pass scan
 * with decoupled look-back that every binning runs): scans two tiles with the
 * first tile's block left out, so the second tile's bounded wait for its
 * predecessor must run out (after about a second) and its block must return.
 * Synchronises `stream` and returns the device status it read and cleared:
 * DCM_ERR_TIMEOUT when the wait ran out as it must. */
int dcm_scan_wait_selftest(dcm_ctx* ctx, dcm_stream_t stream);

/* ---- the hot path ------------------------------------------------------ */

/* Binning, Sections 2.1 and 2.3.  Cell of particle i: cx = floor(x_i / lx),
 * cy = floor(y_i / l), cz = floor(z_i / l) (lx = l unless params.lx is set),
 * computed exactly and clamped to [0, n-1] per axis.  Stable counting
 * sort: particles of one cell keep their input order.
 *   pos        real4[n]       input positions (any order)
 *   cell       int32[n]       out: cell of input particle i
 *   cell_start int32[ncell+1] out: first sorted slot of each cell; cell_start[ncell] = n
 *   perm       int32[n]       out: input index of the particle in sorted slot k
 *   pos_sorted real4[n]       out (nullable): pos[perm[k]]
 * n <= n_max, else DCM_ERR_CAPACITY. */
int dcm_bin(dcm_ctx* ctx, int64_t n, const void* pos, int32_t* cell, int32_t* cell_start,
            int32_t* perm, void* pos_sorted, dcm_stream_t stream);

/* Particle count per density box of edge h (the gray-scale volume's input,
 * Section 2.1).  box_count int32[nboxes] is overwritten. */
int dcm_box_counts(dcm_ctx* ctx, int64_t n, const void* pos, int32_t* box_count, dcm_stream_t stream);

/* Interface detection, Section 2.1 and Eq. 4.  g = box sum of box_count over
 * the (2w+1)^3 periodic neighbourhood; T = integer 2-means threshold of g (or
 * the fixed params.threshold); s = (g >= T), then (params.segmentation = 1)
 * refined by the regularised two-phase segmentation of box_count, then
 * (params.min_component > 0) without its small components
 * (dcm_remove_small_components); iface = s AND some face neighbour has s = 0.  If one phase is empty, T = max(g) + 1 (no
 * interface).
 *   box_count int32[nboxes] in;  s, iface uint8[nboxes] out;
 *   threshold int32[1] out (device);  g int32[nboxes] out (nullable). */
int dcm_detect_interface(dcm_ctx* ctx, const int32_t* box_count, uint8_t* s, uint8_t* iface,
                         int32_t* threshold, int32_t* g, dcm_stream_t stream);

/* Section 2.1's bubble filter: every connected component of s_in (boxes of
 * equal value joined through faces, periodic) with fewer than
 * params.min_component boxes takes the other value; s_out gets the result and
 * iface its interface boxes (as in dcm_detect_interface).  s_in, s_out, iface
 * uint8[nboxes] on the device; s_in and s_out must not overlap.  Needs a
 * context created with params.min_component > 0 (else DCM_ERR_INVALID_ARG).
 * Labelling runs at most 64 hook passes; more raise DCM_ERR_NOT_CONVERGED in
 * the device status.  Asynchronous. */
int dcm_remove_small_components(dcm_ctx* ctx, const uint8_t* s_in, uint8_t* s_out, uint8_t* iface,
                                dcm_stream_t stream);

/* Box-interface distances, Section 2.2 and Algorithm 2.1.  D = 0 on boxes
 * with s = 0 or iface = 1, +inf elsewhere; then Godunov fast-sweeping updates
 * d = min(d, solve(neighbours)) accepted only if <= r_grid, iterated (Jacobi)
 * until no box changes.  Boxes farther than r_grid stay +inf.
 *   D real[nboxes] out;  iters int32[1] out (device, nullable): sweeps used.
 * SYNCHRONOUS: returns DCM_ERR_NOT_CONVERGED if iter_max sweeps did not
 * converge (D then holds the last iterate). */
int dcm_distance(dcm_ctx* ctx, const uint8_t* s, const uint8_t* iface, void* D, int32_t* iters,
                 dcm_stream_t stream);

/* Per-particle cutoffs, Section 2.2.  delta_i = trilinear interpolation of
 * min(D, r_grid) between box centres (k + 1/2) h (periodic);
 * rc_i = clamp(rc_max - (rc_max - rc_min) delta_i / ramp, rc_min, rc_max).
 *   pos real4[n] in; D real[nboxes] in; rc real[n] out. */
int dcm_cutoffs(dcm_ctx* ctx, int64_t n, const void* pos, const void* D, void* rc,
                dcm_stream_t stream);

/* Forces, Section 2.4 and Algorithms 2.2/2.3.  For every particle i:
 *   F_i = sum over j != i with |r_ij| < rc_i (strict; minimum image) of
 *         24 eps_ij [2 (s_ij/r)^12 - (s_ij/r)^6] / r^2 * r_ij,
 *   e_i = 1/2 sum of the same pairs' U = 4 eps_ij [(s_ij/r)^12 - (s_ij/r)^6]
 *         (minus U(rc_i) per pair if shift_energy);
 * no Newton's third law (j's force is not touched from i's loop).
 *   pos_sorted real4[n]     positions sorted by cell (dcm_bin's pos_sorted)
 *   rc         real[n]      cutoff of sorted particle k (values outside
 *                           [0, rc_max], and NaN, are clamped into it)
 *   cell_start int32[ncell+1] from dcm_bin
 *   force      real4[n] out {fx, fy, fz, e_i}
 *   totals     double[3] out (device, nullable): {E, W, accepted pairs}, with
 *              W = 1/2 sum_i sum_j r_ij . F_ij. */
int dcm_forces(dcm_ctx* ctx, int64_t n, const void* pos_sorted, const void* rc,
               const int32_t* cell_start, void* force, double* totals, dcm_stream_t stream);

/* Replace the LJ parameters of ctx (host-side only, validated; takes effect
 * for later calls).  Used when eps and sigma are being optimised. */
int dcm_set_lj(dcm_ctx* ctx, int32_t ntypes, const double* eps, const double* sigma);

/* Adjoint of dcm_forces (differentiation form; the paper has no gradient: this
 * differentiates its force and energy, Section 2.4, with the cutoffs held
 * fixed).  For a scalar loss L(F, E) with upstream dL_dF = dL/dF (real4[n],
 * w ignored) and dL_dE = dL/dE:
 *   dL_dpos[k] = sum_{j in N(k)} [J(r_kj) A_k - dL_dE/2 phi_kj]
 *              + sum_{j : k in N(j)} [-J(r_kj) A_j - dL_dE/2 phi_kj]
 * with N(i) = {j != i : |r_ij| < rc_i}, phi_ij the pair force on i and J its
 * Jacobian (the second sum runs over the particles whose own cutoff reaches
 * k: the stencil's radius is the largest cutoff within the 27 blocks of edge
 * >= 1.001 rc_max around k, found in the context's scratch, so concurrent
 * calls on one context must not overlap).  dL_dparams (device double[2 ntypes],
 * nullable) receives dL/deps_a then dL/dsigma_a, chained through
 * Lorentz-Berthelot mixing.  Inputs as for dcm_forces (sorted order). */
int dcm_forces_backward(dcm_ctx* ctx, int64_t n, const void* pos_sorted, const void* rc, const int32_t* cell_start,
                        const void* dL_dF, double dL_dE, void* dL_dpos, double* dL_dparams, dcm_stream_t stream);

/* Initial evaluation before the first step: bin (state reordered into buffer
 * 1-cur), interface, distances, cutoffs and forces for the current positions;
 * sets t = 0 and thermo.  Synchronous only if distance sweeps need a host
 * check (see dcm_step). */
int dcm_step_init(dcm_ctx* ctx, dcm_state* st, int64_t n, dcm_stream_t stream);

/* nsteps velocity-Verlet timesteps (Section 2; Fig. 3 boxes 1-5):
 *   v += dt/2 F;  x += dt v (wrapped);  bin;
 *   if t % K == 0: box counts, interface, distances, cutoffs;
 *   forces;  v += dt/2 F;  thermo = {E, W, KE, pairs}.
 * Masses are 1.  thermo and the per-particle energies (w of st->force) are
 * those of the call's last timestep; on the cell lists in the mixed form the
 * timesteps before it sum forces only (energy and virial are not evaluated
 * where nothing reads them).  The distance sweeps run in one cooperative
 * launch (bounded grid barriers between sweeps) until a sweep changes
 * nothing, at most params.iter_max sweeps; non-convergence, or a barrier wait
 * that ran out (DCM_ERR_TIMEOUT), is reported by dcm_status().
 * With params.skin == 0 the call never waits on the host.  With skin > 0
 * (Verlet lists) each step reads the largest displacement back to the host
 * to decide whether to rebin and rebuild the lists (so it synchronises the
 * stream once per step, may grow the list storage, and leaves the state in
 * buffer cur unchanged on steps without a rebuild; between rebuilds positions
 * are not wrapped into the box). */
int dcm_step(dcm_ctx* ctx, dcm_state* st, int64_t n, double dt, int32_t nsteps, dcm_stream_t stream);

/* Same result as dcm_distance, for callers that cannot allocate device
 * memory: code whose device memory belongs to another allocator or
 * framework, or a plugin that is only handed device buffers.  It needs no
 * dcm_ctx (whose creation allocates) and calls no allocating routine.  The
 * paper has no counterpart: this is a deployment variant of the same fast
 * sweeping.
 *   p      host pointer to the parameters (validated as by dcm_validate_params)
 *   s, iface, D, iters: as for dcm_distance (device pointers; iters nullable)
 * Scratch: one fixed 8 MiB device array compiled into the library (held by
 * every GPU that loads it, until exit), holding the second Jacobi iterate
 * (nboxes reals) and iter_max + 2 change flags; a grid or iter_max needing more
 * returns DCM_ERR_CAPACITY before any launch (e.g. up to about 2.0M boxes in
 * the mixed form, 1.0M in FP64).  The first call on each device looks up the
 * array's device address with cudaGetSymbolAddress (device current) and
 * caches it per device index: `stream` must belong to the current device, and
 * a cudaDeviceReset invalidates the cached address (do not call this entry
 * point on a device after resetting it).  Every call shares the array: calls
 * whose kernels may overlap on the GPU race.
 * SYNCHRONOUS like dcm_distance (it waits on the stream between chunks of
 * sweeps); returns DCM_ERR_NOT_CONVERGED likewise, D then holding the last
 * iterate and *iters = -1. */
int dcm_distance_noalloc(const dcm_params* p, const uint8_t* s, const uint8_t* iface, void* D, int32_t* iters,
                         dcm_stream_t stream);

/* ---- batched form: many independent systems, two launches per timestep ---- */

/* R independent replicas (the batching form) that share every
 * parameter in *p except the box and the particle count: replica r has box
 * boxes[3r .. 3r+2] (host) and counts[r] particles (host).  Each replica is
 * validated as a single system (dcm_validate_params).  The state arrays of
 * dcm_state are the concatenation of the replicas: replica r owns slots
 * [offset[r], offset[r+1]) (dcm_batch_offsets) and its particles stay there;
 * thermo is double[4 R] = {E, W, KE, pairs} per replica, of the last
 * timestep of a dcm_batch_step call (the timesteps before it evaluate forces
 * only and run no thermo stage).  By default a whole
 * timestep of all replicas is two persistent cooperative launches (the
 * persistent plan): binning and recomputation, then forces, kick and thermo;
 * the stages inside each are separated by grid-wide barriers, and the force
 * stage pulls (replica, tile) work items of 32 particles from a device queue
 * (Section 2.4's dynamic tasks).  dcm_batch_set_persistent(b, 0)
 * selects the per-stage plan instead (each stage launched over all
 * replicas; a force launch of at most 16 waves of blocks takes its tiles
 * widest cutoff first, after three small launches that order them).
 * Per-replica boxes, grids, thresholds and reductions are read
 * from a device table in both plans.  The batched form steps over
 * cell lists: p->skin must be 0, and p->min_component 0 (no bubble filter).
 * Synchronous; allocates. */
typedef struct dcm_batch dcm_batch;
int dcm_batch_create(const dcm_params* p, int32_t R, const double* boxes, const int64_t* counts, dcm_batch** out);
void dcm_batch_destroy(dcm_batch* b);
const char* dcm_batch_last_error(const dcm_batch* b);

/* offsets (host, R+1 entries): first slot of every replica and the total. */
int dcm_batch_offsets(const dcm_batch* b, int64_t* offsets);

/* Threads per block of the batched force kernel: 64, 128 (default) or 256
 * (set by the autotuner).  Invalidates a captured graph. */
int dcm_batch_set_force_block(dcm_batch* b, int32_t threads);

/* As dcm_step_init / dcm_step for all replicas at once (asynchronous; the
 * distance sweeps run until a sweep changes nothing, at most
 * params.iter_max, and report non-convergence through dcm_batch_status).  In the persistent plan a barrier wait that runs past
 * the wait budget (dcm_batch_set_wait_budget) ends the launch and records
 * DCM_ERR_TIMEOUT in the batch's device status; the step's results are then
 * undefined. */
int dcm_batch_step_init(dcm_batch* b, dcm_state* st, dcm_stream_t stream);
int dcm_batch_step(dcm_batch* b, dcm_state* st, double dt, int32_t nsteps, dcm_stream_t stream);

/* Capture one recomputation period (K steps, or 2K if K is odd so that the
 * double buffers return to the same side) of dcm_batch_step into a CUDA graph
 * on `stream` (must not be the legacy default stream); st->t must be a
 * multiple of K.  The graph is bound to st's buffers.  Nothing is executed. */
int dcm_batch_capture(dcm_batch* b, dcm_state* st, double dt, dcm_stream_t stream);

/* 1 (default): the persistent plan, two cooperative launches per timestep;
 * 0: the per-stage plan.  Both give the same results (bit for bit, except
 * for the order of floating-point atomics, which neither plan uses).
 * Invalidates a captured graph. */
int dcm_batch_set_persistent(dcm_batch* b, int32_t on);

/* The DCM_ACC_* form of the batched force stage, written to *form: the
 * context rule of dcm_accumulation, then DCM_ACC_PLANE_FP64 for every FP64
 * form and DCM_ACC_PLANE_KAHAN for every other compensated one (the batched
 * form runs the plain and the plane forms).  Host only. */
int dcm_batch_accumulation(const dcm_batch* b, int32_t* form);

/* Particles per work item of the persistent plan's force queue: a multiple
 * of 32 in 32 .. 4096 (default 32; set by the autotuner).  Each item lies in
 * one replica; a warp takes one item at a time.  Invalidates a captured
 * graph. */
int dcm_batch_set_tile(dcm_batch* b, int32_t particles);

/* Longest time, in nanoseconds (>= 1000), that a block of the persistent
 * plan waits at a grid barrier before it gives up with DCM_ERR_TIMEOUT.
 * Default 2 s.  Invalidates a captured graph. */
int dcm_batch_set_wait_budget(dcm_batch* b, int64_t ns);

/* Self-test of the persistent plan's failure path: launches the persistent
 * grid with one barrier that waits for `phantom` (> 0) blocks that do not
 * exist, so every wait must run out after budget_ns (1000 .. 1e10)
 * nanoseconds and every block must return.  Synchronises `stream` and returns
 * the device status it read and cleared: DCM_ERR_TIMEOUT when the waits ran
 * out as they must (phantom = 0: DCM_OK). */
int dcm_batch_barrier_selftest(dcm_batch* b, int32_t phantom, int64_t budget_ns, dcm_stream_t stream);

/* Launch the captured graph ngraphs times (st->t advances by
 * ngraphs * dcm_batch_graph_steps).  st must hold the captured buffers. */
int dcm_batch_replay(dcm_batch* b, dcm_state* st, int32_t ngraphs, dcm_stream_t stream);
int dcm_batch_graph_steps(const dcm_batch* b);

/* As dcm_status, dcm_set_timing, dcm_stage_times, dcm_launch_count.  In the
 * persistent plan the stage times come from a clock inside the launch: block
 * 0 reads the GPU's global timer as it leaves each grid barrier and charges
 * the interval to the stage that just ended. */
int dcm_batch_status(dcm_batch* b, dcm_stream_t stream);
int dcm_batch_set_timing(dcm_batch* b, int32_t capacity);
int dcm_batch_stage_times(dcm_batch* b, double* ms, int64_t* count);
int dcm_batch_launch_count(dcm_batch* b, int64_t* count, int32_t reset);

/* ---- instrumentation -------------------------------------------------- */

/* Stages of dcm_step whose GPU time can be measured. */
enum dcm_stage {
  DCM_STAGE_KICK_DRIFT = 0, /* half kick, drift, cell count */
  DCM_STAGE_BIN = 1,        /* scan, scatter, per-cell sort, gather of the state */
  DCM_STAGE_DETECT = 2,     /* dcm_detect_interface */
  DCM_STAGE_DISTANCE = 3,   /* dcm_distance sweeps */
  DCM_STAGE_CUTOFFS = 4,    /* dcm_cutoffs */
  DCM_STAGE_FORCES = 5,     /* dcm_forces kernel (without the final reduction) */
  DCM_STAGE_KICK = 6,       /* second half kick and kinetic energy */
  DCM_STAGE_LISTS = 7,      /* Verlet list build (params.skin > 0) */
  DCM_NSTAGES = 8
};

/* capacity > 0: every later stage run on ctx records a CUDA event pair on the
 * launching stream around the stage, for up to `capacity` runs per stage
 * between two dcm_stage_times calls (events are created here, which
 * synchronises the device when the table grows); capacity = 0 turns timing
 * off (the default after dcm_create).  Clears the record. */
int dcm_set_timing(dcm_ctx* ctx, int32_t capacity);

/* SYNCHRONOUS (device-wide): ms[s] receives the summed GPU time of stage s
 * over the event pairs recorded since the last call and count[s] how many
 * stage runs there were (either pointer may be NULL); the record is then
 * cleared.  Returns DCM_ERR_CAPACITY if more runs than the capacity happened
 * (ms then covers the first `capacity` runs only). */
int dcm_stage_times(dcm_ctx* ctx, double* ms, int64_t* count);

/* Number of CUDA kernels this context has launched; reset if reset != 0. */
int dcm_launch_count(dcm_ctx* ctx, int64_t* count, int32_t reset);

/* The DCM_FORCE_* kernel that dcm_forces and dcm_step run on the cell lists
 * for this context's parameters (params.force_kernel with AUTO and the
 * kernels' limits resolved), written to *kernel.  Host only. */
int dcm_force_kernel(const dcm_ctx* ctx, int32_t* kernel);

/* The DCM_ACC_* form in which this context's force launches sum each
 * particle's pair terms (params.accumulation with AUTO and the kernels'
 * limits resolved; DCM_ACC_FP32 for the FP64 precision form, whose sums are
 * FP64), written to *form.  Host only. */
int dcm_accumulation(const dcm_ctx* ctx, int32_t* form);

#ifdef __cplusplus
}
#endif

#endif /* DCM_H */
