"""FP64 CPU oracle for the Dynamic Cutoff Method's per-timestep path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
C-ABI library and its Python binding) never imports, links or runs anything
here, and this package imports nothing from the product.

Thin numpy wrappers around ``dcm_oracle.c`` (plain sequential double
precision), plus the composed pipeline of one timestep:

  bin (Sec. 2.1, 2.3) -> gray-scale volume and 2-means segmentation (Sec. 2.1,
  Eq. 4) -> interface boxes -> CFSM distances (Sec. 2.2, Alg. 2.1) ->
  trilinear distance and cutoff rule (Sec. 2.2) -> i-centric LJ forces
  without Newton's third law (Sec. 2.4, Alg. 2.2/2.3) -> velocity Verlet.

Readings of points the paper leaves open are fixed in the function docstrings
(smoothing half-width, 2-means threshold, liquid-side interface boxes,
r_grid = ramp + 2h, linear cutoff ramp, unshifted energy).

Pinned by tests/test_oracle_pins.py against closed forms, brute force,
invariances and textbook special cases.  ``adjoint`` is pinned by central
finite differences of the oracle's own forward pass and by a dense
autograd formulation.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dcm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle in-tree with gcc (no FMA contraction, no -march)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            I64, I32, D = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "orc_cell_coord": (I64, [D, D, I64]),
                "orc_bin": (None, [I64, _f64p, _f64p, _i64p, _i32p, _i32p, _i32p, _i32p]),
                "orc_smooth": (None, [_i32p, _i64p, I32, _i32p]),
                "orc_two_means": (I64, [_i32p, I64, I32]),
                "orc_segment": (None, [_i32p, _i64p, I64, _u8p, _u8p]),
                "orc_interface": (None, [_u8p, _i64p, _u8p]),
                "orc_remove_small_components": (I64, [_u8p, _i64p, I64, _u8p]),
                "orc_ms_segment": (I32, [_i32p, _i64p, D, I32, I32, _u8p, _f64p, _f64p]),
                "orc_cfsm": (I32, [_u8p, _u8p, _i64p, D, D, I32, _f64p]),
                "orc_distance_jacobi": (I32, [_u8p, _u8p, _i64p, D, D, I32, _f64p]),
                "orc_distance_sweep8": (I32, [_u8p, _u8p, _i64p, D, D, I32, _f64p]),
                "orc_cutoffs": (None, [I64, _f64p, _f64p, _i64p, D, D, D, D, D, _f64p, _f64p]),
                "orc_cutoff_rule": (D, [D, D, D, D]),
                "orc_forces_brute": (None, [I64, _f64p, _i32p, _f64p, _f64p, I32, _f64p, _f64p, I32,
                                            _f64p, _f64p, _f64p, _i64p]),
                "orc_forces_cells": (None, [I64, _f64p, _i32p, _f64p, _f64p, _f64p, _i64p, I32, _f64p,
                                            _f64p, I32, I32, _f64p, _f64p, _f64p, _i64p]),
                "orc_forces_subset": (None, [I64, _f64p, _i32p, _f64p, _f64p, _f64p, _i64p, I32, _f64p, _f64p,
                                             I32, I64, _i64p, I32, _f64p, _f64p, _f64p, _i64p]),
                "orc_adjoint_brute": (None, [I64, _f64p, _i32p, _f64p, _f64p, I32, _f64p, _f64p, I32, _f64p, D,
                                             _f64p, _f64p, _f64p]),
                "orc_kick": (None, [I64, _f64p, _f64p, D]),
                "orc_drift": (None, [I64, _f64p, _f64p, D, _f64p]),
                "orc_kinetic": (D, [I64, _f64p]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _vec3(v):
    return np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), (3,)))


def grid_dims(box, edge) -> np.ndarray:
    """Number of boxes per dimension; the box must be an integer multiple of the
    edge (one edge for all three axes, or one per axis)."""
    n = []
    for L, e in zip(box, _vec3(edge)):
        k = int(round(L / e))
        if k < 1 or abs(k * e - L) > 1e-9 * L:
            raise ValueError(f"box length {L} is not a multiple of edge {e}")
        n.append(k)
    return np.asarray(n, dtype=np.int64)


# --------------------------------------------------------------------------
# Binning
# --------------------------------------------------------------------------
def bin_particles(pos, box, l):
    """Stable counting sort by cell (Sections 2.1, 2.3).

    Returns (cell[N], count[ncell], start[ncell+1], perm[N]) as int32, with the
    cell of a particle c = cx + nx (cy + ny cz), cx = floor(x / l_x) exactly
    (l one edge for all axes or a per-axis triple).
    """
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    nc = grid_dims(box, l)
    ncell = int(np.prod(nc))
    cell = np.empty(max(n, 1), np.int32)
    count = np.empty(ncell, np.int32)
    start = np.empty(ncell + 1, np.int32)
    perm = np.empty(max(n, 1), np.int32)
    _load().orc_bin(n, _p(pos, _f64p), _p(_vec3(l), _f64p), _p(nc, _i64p), _p(cell, _i32p),
                    _p(count, _i32p), _p(start, _i32p), _p(perm, _i32p))
    return cell[:n], count, start, perm[:n]


def cell_coord(x: float, l: float, n: int) -> int:
    return int(_load().orc_cell_coord(float(x), float(l), int(n)))


# --------------------------------------------------------------------------
# Interface detection
# --------------------------------------------------------------------------
def smooth(count, nh, w: int = 2):
    """Gray-scale value of every box: sum of particle counts over the
    (2w+1)^3 periodic neighbourhood (reading: w = 2 suppresses Poisson noise
    that the paper's length term and bubble filter would remove)."""
    nh = np.asarray(nh, dtype=np.int64)
    count = np.ascontiguousarray(count, dtype=np.int32)
    g = np.empty(int(np.prod(nh)), np.int32)
    _load().orc_smooth(_p(count, _i32p), _p(nh, _i64p), int(w), _p(g, _i32p))
    return g


def two_means(g, max_iter: int = 64) -> int:
    """Integer 2-means threshold T (s = g >= T); T = g_max + 1 when a phase is empty."""
    g = np.ascontiguousarray(g, dtype=np.int32)
    return int(_load().orc_two_means(_p(g, _i32p), g.size, max_iter))


def segment(g, nh, T: int):
    """Segmented volume S (Eq. 4) and liquid-side interface boxes."""
    nh = np.asarray(nh, dtype=np.int64)
    g = np.ascontiguousarray(g, dtype=np.int32)
    s = np.empty(g.size, np.uint8)
    iface = np.empty(g.size, np.uint8)
    _load().orc_segment(_p(g, _i32p), _p(nh, _i64p), int(T), _p(s, _u8p), _p(iface, _u8p))
    return s, iface


def interface(s, nh):
    """Liquid-side interface boxes of a segmented volume S."""
    nh = np.asarray(nh, dtype=np.int64)
    s = np.ascontiguousarray(s, dtype=np.uint8)
    iface = np.empty(s.size, np.uint8)
    _load().orc_interface(_p(s, _u8p), _p(nh, _i64p), _p(iface, _u8p))
    return iface


def remove_small_components(s, nh, min_boxes: int):
    """Section 2.1's bubble filter (reading): every face-connected periodic
    component of either phase with fewer than ``min_boxes`` boxes takes the
    other value.  Returns (s_filtered, number of flipped components)."""
    nh = np.asarray(nh, dtype=np.int64)
    s = np.ascontiguousarray(s, dtype=np.uint8)
    out = np.empty_like(s)
    k = _load().orc_remove_small_components(_p(s, _u8p), _p(nh, _i64p), int(min_boxes), _p(out, _u8p))
    return out, int(k)


def ms_segment(count, nh, s0, nu: float, inner: int, outer: int):
    """Section 2.1's regularised two-phase Mumford-Shah segmentation of the
    box counts (reading and iteration in dcm_oracle.c), from the volume s0.
    Returns (s, u, (c0, c1), outer iterations run)."""
    nh = np.asarray(nh, dtype=np.int64)
    g = np.ascontiguousarray(count, dtype=np.int32)
    s = np.array(s0, dtype=np.uint8, copy=True)
    u = np.zeros(g.size, dtype=np.float64)
    c = np.zeros(2, dtype=np.float64)
    k = _load().orc_ms_segment(_p(g, _i32p), _p(nh, _i64p), float(nu), int(inner), int(outer), _p(s, _u8p),
                               _p(u, _f64p), _p(c, _f64p))
    return s, u, (float(c[0]), float(c[1])), int(k)


def ms_energy(count, nh, s, c0, c1, nu):
    """The functional E(s; c0, c1) of the segmentation reading: squared
    deviations from the phase values plus nu times the faces between phases."""
    nh = np.asarray(nh, dtype=np.int64)
    g = np.asarray(count, dtype=np.float64).reshape(nh[2], nh[1], nh[0])
    sv = np.asarray(s, dtype=np.float64).reshape(nh[2], nh[1], nh[0])
    data = (sv * (g - c1) ** 2 + (1.0 - sv) * (g - c0) ** 2).sum()
    faces = sum(np.abs(np.roll(sv, -1, axis=a) - sv).sum() for a in range(3))
    return float(data + nu * faces)


def detect_interface(count, nh, w: int = 2, threshold=None, min_component: int = 0, ms=None):
    """count -> (g, T, s, iface).  ``threshold`` fixes T instead of 2-means;
    ``ms = (nu, inner, outer)`` refines S by the regularised Mumford-Shah
    segmentation of the unsmoothed counts, starting from the threshold's S;
    ``min_component > 0`` removes smaller components of either phase from S
    before the interface boxes are taken."""
    g = smooth(count, nh, w)
    T = two_means(g) if threshold is None else int(threshold)
    s, iface = segment(g, nh, T)
    if ms is not None:
        s, _, _, _ = ms_segment(count, nh, s, *ms)
        iface = interface(s, nh)
    if min_component > 0:
        s, _ = remove_small_components(s, nh, min_component)
        iface = interface(s, nh)
    return g, T, s, iface


# --------------------------------------------------------------------------
# Distances
# --------------------------------------------------------------------------
def _distance(fn, s, iface, nh, h, r_grid, iter_max):
    nh = np.asarray(nh, dtype=np.int64)
    s = np.ascontiguousarray(s, dtype=np.uint8)
    iface = np.ascontiguousarray(iface, dtype=np.uint8)
    D = np.empty(s.size, np.float64)
    it = fn(_p(s, _u8p), _p(iface, _u8p), _p(nh, _i64p), float(h), float(r_grid), int(iter_max), _p(D, _f64p))
    return D, int(it)


def cfsm(s, iface, nh, h, r_grid, iter_max: int = 1000):
    """Algorithm 2.1 (queue-based cutoff fast sweeping); returns (D, passes)."""
    return _distance(_load().orc_cfsm, s, iface, nh, h, r_grid, iter_max)


def distance_jacobi(s, iface, nh, h, r_grid, iter_max: int = 1000):
    return _distance(_load().orc_distance_jacobi, s, iface, nh, h, r_grid, iter_max)


def distance_sweep8(s, iface, nh, h, r_grid, iter_max: int = 1000):
    return _distance(_load().orc_distance_sweep8, s, iface, nh, h, r_grid, iter_max)


# --------------------------------------------------------------------------
# Cutoffs
# --------------------------------------------------------------------------
def cutoffs(pos, D, nh, h, r_grid, rc_min, rc_max, ramp):
    """Per-particle delta_i (trilinear) and rc_i (linear ramp reading)."""
    pos = _f64(pos).reshape(-1, 3)
    nh = np.asarray(nh, dtype=np.int64)
    D = _f64(D)
    n = pos.shape[0]
    delta = np.empty(max(n, 1))
    rc = np.empty(max(n, 1))
    _load().orc_cutoffs(n, _p(pos, _f64p), _p(D, _f64p), _p(nh, _i64p), float(h), float(r_grid),
                        float(rc_min), float(rc_max), float(ramp), _p(delta, _f64p), _p(rc, _f64p))
    return delta[:n], rc[:n]


def cutoff_rule(delta, rc_min, rc_max, ramp):
    return _load().orc_cutoff_rule(float(delta), float(rc_min), float(rc_max), float(ramp))


# --------------------------------------------------------------------------
# Forces
# --------------------------------------------------------------------------
@dataclass
class ForceResult:
    F: np.ndarray       # (N, 3)
    e: np.ndarray       # (N,) per-particle energy (half of each pair's U)
    E: float
    W: float
    npairs: int


def _lj_arrays(eps, sigma):
    eps = np.ascontiguousarray(np.atleast_1d(eps), dtype=np.float64)
    sigma = np.ascontiguousarray(np.atleast_1d(sigma), dtype=np.float64)
    if eps.size != sigma.size or eps.size < 1 or eps.size > 4:
        raise ValueError("eps and sigma must have the same length (1..4 types)")
    return eps, sigma


def forces_brute(pos, rc, box, types=None, eps=(1.0,), sigma=(1.0,), shift=False) -> ForceResult:
    """O(N^2) forces with per-particle cutoffs (Algorithm 2.3 over all j)."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    rc = _f64(np.broadcast_to(rc, (n,)))
    eps, sigma = _lj_arrays(eps, sigma)
    t = None if types is None else np.ascontiguousarray(types, dtype=np.int32)
    F = np.empty((max(n, 1), 3))
    e = np.empty(max(n, 1))
    out = np.empty(2)
    npairs = ctypes.c_int64(0)
    _load().orc_forces_brute(n, _p(pos, _f64p), None if t is None else _p(t, _i32p), _p(rc, _f64p),
                             _p(_vec3(box), _f64p), eps.size, _p(eps, _f64p), _p(sigma, _f64p), int(shift),
                             _p(F, _f64p), _p(e, _f64p), _p(out, _f64p), ctypes.byref(npairs))
    return ForceResult(F[:n], e[:n], float(out[0]), float(out[1]), int(npairs.value))


def forces_cells(pos, rc, box, l, types=None, eps=(1.0,), sigma=(1.0,), shift=False,
                 nthreads: int = 1) -> ForceResult:
    """Cell-list forces (Algorithms 2.2 + 2.3), OpenMP dynamic(20) over i."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    rc = _f64(np.broadcast_to(rc, (n,)))
    eps, sigma = _lj_arrays(eps, sigma)
    nc = grid_dims(box, l)
    t = None if types is None else np.ascontiguousarray(types, dtype=np.int32)
    F = np.empty((max(n, 1), 3))
    e = np.empty(max(n, 1))
    out = np.empty(2)
    npairs = ctypes.c_int64(0)
    _load().orc_forces_cells(n, _p(pos, _f64p), None if t is None else _p(t, _i32p), _p(rc, _f64p),
                             _p(_vec3(box), _f64p), _p(_vec3(l), _f64p), _p(nc, _i64p), eps.size,
                             _p(eps, _f64p), _p(sigma, _f64p), int(shift), int(nthreads),
                             _p(F, _f64p), _p(e, _f64p), _p(out, _f64p), ctypes.byref(npairs))
    return ForceResult(F[:n], e[:n], float(out[0]), float(out[1]), int(npairs.value))


def forces_subset(pos, rc, box, l, idx, types=None, eps=(1.0,), sigma=(1.0,), shift=False, nthreads: int = 1):
    """Cell-list forces of the particles idx only: (F[m,3], e[m], w[m], npairs[m]),
    with e and w each particle's half-pair energy and virial sums."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    rc = _f64(np.broadcast_to(rc, (n,)))
    eps, sigma = _lj_arrays(eps, sigma)
    nc = grid_dims(box, l)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    m = idx.size
    t = None if types is None else np.ascontiguousarray(types, dtype=np.int32)
    F = np.empty((max(m, 1), 3))
    e = np.empty(max(m, 1))
    w = np.empty(max(m, 1))
    npairs = np.empty(max(m, 1), np.int64)
    _load().orc_forces_subset(n, _p(pos, _f64p), None if t is None else _p(t, _i32p), _p(rc, _f64p),
                              _p(_vec3(box), _f64p), _p(_vec3(l), _f64p), _p(nc, _i64p), eps.size, _p(eps, _f64p),
                              _p(sigma, _f64p), int(shift), m, _p(idx, _i64p), int(nthreads), _p(F, _f64p),
                              _p(e, _f64p), _p(w, _f64p), _p(npairs, _i64p))
    return F[:m], e[:m], w[:m], npairs[:m]


def adjoint(pos, rc, box, A, dLdE, types=None, eps=(1.0,), sigma=(1.0,), shift=False):
    """Gradient of a loss L(F, E) with respect to positions and per-type LJ
    parameters, cutoffs held fixed (O(N^2), FP64).  A = dL/dF (N x 3),
    dLdE = dL/dE.  Returns (dL/dpos (N x 3), dL/deps (ntypes), dL/dsigma
    (ntypes)); the type-pair sums are chained through Lorentz-Berthelot
    mixing, eps_ab = sqrt(eps_a eps_b), sigma_ab = (sigma_a + sigma_b) / 2."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    rc = _f64(np.broadcast_to(rc, (n,)))
    A = _f64(A).reshape(-1, 3)
    eps, sigma = _lj_arrays(eps, sigma)
    nt = eps.size
    t = None if types is None else np.ascontiguousarray(types, dtype=np.int32)
    G = np.empty((max(n, 1), 3))
    dep = np.empty(nt * nt)
    dsp = np.empty(nt * nt)
    _load().orc_adjoint_brute(n, _p(pos, _f64p), None if t is None else _p(t, _i32p), _p(rc, _f64p),
                              _p(_vec3(box), _f64p), nt, _p(eps, _f64p), _p(sigma, _f64p), int(shift),
                              _p(A, _f64p), float(dLdE), _p(G, _f64p), _p(dep, _f64p), _p(dsp, _f64p))
    de, ds = mix_chain(dep, dsp, eps)
    return G[:n], de, ds


def mix_chain(deps_pair, dsig_pair, eps):
    """Chain per-type-pair parameter gradients to per-type gradients through
    eps_ab = sqrt(eps_a eps_b) and sigma_ab = (sigma_a + sigma_b) / 2."""
    eps = np.asarray(eps, np.float64)
    nt = eps.size
    de = np.zeros(nt)
    ds = np.zeros(nt)
    for a in range(nt):
        for b in range(nt):
            p = a * nt + b
            if a == b:
                de[a] += deps_pair[p]
                ds[a] += dsig_pair[p]
            else:
                de[a] += deps_pair[p] * 0.5 * math.sqrt(eps[b] / eps[a])
                de[b] += deps_pair[p] * 0.5 * math.sqrt(eps[a] / eps[b])
                ds[a] += 0.5 * dsig_pair[p]
                ds[b] += 0.5 * dsig_pair[p]
    return de, ds


def lj_pair(r, eps=1.0, sigma=1.0):
    """Closed-form 12-6 LJ: (U(r), |F|(r) along r_hat).  Plain numpy."""
    sr6 = (sigma / r) ** 6
    return 4 * eps * (sr6 * sr6 - sr6), 24 * eps * (2 * sr6 * sr6 - sr6) / r


# --------------------------------------------------------------------------
# Parameters and the composed timestep
# --------------------------------------------------------------------------
@dataclass
class Params:
    box: tuple
    h: float = 1.5            # density-grid box edge (Section 2.1)
    l: float = 1.5            # force-cell edge (Section 2.3; l <= rc_min)
    rc_min: float = 3.0
    rc_max: float = 6.0
    ramp: float = None        # delta at which rc reaches rc_min; default rc_max - rc_min
    r_grid: float = None      # CFSM threshold; default ramp + 2h
    smooth_w: int = 2
    threshold: int = None     # fixed T instead of 2-means
    iter_max: int = 1000
    eps: tuple = (1.0,)
    sigma: tuple = (1.0,)
    shift: bool = False
    recompute_every: int = 1  # K: interface/distance/cutoffs every K steps
    min_component: int = 0    # > 0: remove smaller components of S (Section 2.1's bubble filter)

    def __post_init__(self):
        if self.ramp is None:
            self.ramp = self.rc_max - self.rc_min
        if self.r_grid is None:
            self.r_grid = self.ramp + 2.0 * self.h


def assign_cutoffs(pos, p: Params):
    """Interface detection + CFSM + cutoffs for current positions.
    Returns dict(count, g, T, s, iface, D, passes, delta, rc)."""
    nh = grid_dims(p.box, p.h)
    _, count, _, _ = bin_particles(pos, p.box, p.h)
    g, T, s, iface = detect_interface(count, nh, p.smooth_w, p.threshold, p.min_component)
    D, passes = cfsm(s, iface, nh, p.h, p.r_grid, p.iter_max)
    delta, rc = cutoffs(pos, D, nh, p.h, p.r_grid, p.rc_min, p.rc_max, p.ramp)
    return dict(count=count, g=g, T=T, s=s, iface=iface, D=D, passes=passes, delta=delta, rc=rc)


def forces(pos, rc, p: Params, types=None, nthreads: int = 1) -> ForceResult:
    return forces_cells(pos, rc, p.box, p.l, types, p.eps, p.sigma, p.shift, nthreads)


def kick(vel, F, half_dt):
    vel = _f64(vel).reshape(-1, 3).copy()
    F = _f64(F).reshape(-1, 3)
    _load().orc_kick(vel.shape[0], _p(vel, _f64p), _p(F, _f64p), float(half_dt))
    return vel


def drift(pos, vel, dt, box):
    pos = _f64(pos).reshape(-1, 3).copy()
    vel = _f64(vel).reshape(-1, 3)
    _load().orc_drift(pos.shape[0], _p(pos, _f64p), _p(vel, _f64p), float(dt), _p(_vec3(box), _f64p))
    return pos


def kinetic(vel) -> float:
    vel = _f64(vel).reshape(-1, 3)
    return float(_load().orc_kinetic(vel.shape[0], _p(vel, _f64p)))


@dataclass
class State:
    pos: np.ndarray
    vel: np.ndarray
    rc: np.ndarray
    F: np.ndarray
    E: float
    W: float
    t: int = 0


def init_state(pos, vel, p: Params, types=None, nthreads: int = 1) -> State:
    """Cutoffs from the initial positions plus the first force evaluation."""
    pos = _f64(pos).reshape(-1, 3).copy()
    vel = _f64(vel).reshape(-1, 3).copy()
    rc = assign_cutoffs(pos, p)["rc"]
    fr = forces(pos, rc, p, types, nthreads)
    return State(pos, vel, rc, fr.F, fr.E, fr.W, 0)


def step(st: State, dt: float, p: Params, types=None, nthreads: int = 1) -> State:
    """One velocity-Verlet timestep (Fig. 3, boxes 1-5): half kick, drift,
    cutoffs every K steps (counted from the initial evaluation), forces, half kick."""
    vel = kick(st.vel, st.F, 0.5 * dt)
    pos = drift(st.pos, vel, dt, p.box)
    t = st.t + 1
    rc = assign_cutoffs(pos, p)["rc"] if t % p.recompute_every == 0 else st.rc
    fr = forces(pos, rc, p, types, nthreads)
    vel = kick(vel, fr.F, 0.5 * dt)
    return State(pos, vel, rc, fr.F, fr.E, fr.W, t)
