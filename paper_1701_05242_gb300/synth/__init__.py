"""Seeded synthetic inputs: liquid/vapor Lennard-Jones slabs in reduced units.

This module only generates inputs (positions, types, velocities, slab
geometry).  It holds none of the dynamic-cutoff method's arithmetic, and both
the FP64 oracle and the CUDA path consume the arrays it returns, so the two
sides start from bit-identical FP32 states.

Recipe (all seeded, deterministic):
  * Geometry: periodic box (Lx, Ly, Lz); the liquid slab fills the central
    third in z (the planar system of the paper's Section 3, Fig. 5a), the vapor
    the rest.  Or (``cylinder_radius > 0``) a liquid cylinder of that radius
    along x with its axis at (Ly/2, Lz/2) (the curved interface of Fig. 5b).
    Particle counts are N_phase = floor(rho * V_phase + 0.5).
  * Optional capillary waves on each of the two surfaces: 16 modes
    (1 <= kx, ky <= 4), amplitude proportional to 1/|k|, random phases, scaled
    so that the largest excursion over the xy plane equals ``wave_amp``.
  * Positions: random sequential addition (uniform proposals, rejected if
    closer than d_min = 0.85 to an already placed particle), liquid first.
  * Velocities: Maxwell-Boltzmann at T*, centre-of-mass velocity removed, then
    rescaled so the kinetic temperature with 3N-3 degrees of freedom is T*.
  * Types (optional): exactly half the particles (rounded down) get type 1,
    chosen by a seeded permutation.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsa.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator's C code in-tree (plain gcc, no -march flags)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d = ctypes.c_double
            pd = ctypes.POINTER(ctypes.c_double)
            lib.synth_rsa_slab.restype = ctypes.c_int
            pi64 = ctypes.POINTER(ctypes.c_int64)
            lib.synth_rsa_slab.argtypes = [d, d, d, ctypes.c_int, pi64, pi64, d, ctypes.c_uint64,
                                           ctypes.c_int, pd, pd, pd, pd, d,
                                           ctypes.c_int, pd, pd, pd, pd, d,
                                           ctypes.c_int64, ctypes.POINTER(ctypes.c_float)]
            lib.synth_rsa_cylinder.restype = ctypes.c_int
            lib.synth_rsa_cylinder.argtypes = [d, d, d, ctypes.c_int, pi64, pi64, d, ctypes.c_uint64, d, d, d,
                                               ctypes.c_int64, ctypes.POINTER(ctypes.c_float)]
            lib.synth_uniform.restype = None
            lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, pd]
            _lib = lib
    return _lib


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n counter-based U[0,1) doubles of stream ``seed`` (SplitMix64)."""
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniform(seed, offset, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


@dataclass
class SlabSpec:
    """Geometry and thermodynamic state of one synthetic slab."""
    box: tuple
    rho_l: float = 0.8
    rho_v: float = 0.02
    temperature: float = 0.7
    liquid_fraction: float = 1.0 / 3.0
    wave_amp: float = 0.0
    ntypes: int = 1
    d_min: float = 0.85
    seed: int = 0
    name: str = ""
    cylinder_radius: float = 0.0

    @property
    def liquid_volume(self) -> float:
        if self.cylinder_radius > 0:
            return math.pi * self.cylinder_radius ** 2 * self.box[0]
        z0, z1 = self.liquid_bounds
        return self.box[0] * self.box[1] * (z1 - z0)

    @property
    def liquid_bounds(self):
        lz = self.box[2]
        t = self.liquid_fraction * lz
        z0 = 0.5 * (lz - t)
        return z0, z0 + t

    @property
    def n_liquid(self) -> int:
        return int(math.floor(self.rho_l * self.liquid_volume + 0.5))

    @property
    def n_vapor(self) -> int:
        v = self.box[0] * self.box[1] * self.box[2] - self.liquid_volume
        return int(math.floor(self.rho_v * v + 0.5))

    @property
    def n(self) -> int:
        return self.n_liquid + self.n_vapor


def named(name: str) -> SlabSpec:
    """The named workloads: sizes follow the liquid/vapor slab systems."""
    if name == "slab_1935":          # 12x12x48, N = 1,935, one force eval + 100 NVE steps
        return SlabSpec(box=(12.0, 12.0, 48.0), name=name)
    if name == "slab_1m":            # 96x96x384, N = 990,904
        return SlabSpec(box=(96.0, 96.0, 384.0), name=name)
    if name == "slab_16m":           # 240x240x960, N = 15,482,880, capillary waves 2.0 sigma
        return SlabSpec(box=(240.0, 240.0, 960.0), wave_amp=2.0, name=name)
    if name == "slab_8m":            # 180x180x960, N = 8,709,120, capillary waves 2.0 sigma (profiling size)
        return SlabSpec(box=(180.0, 180.0, 960.0), wave_amp=2.0, name=name)
    if name == "slab_256k_2types":   # 61.5x61.5x246, N = 260,522, two LJ types
        return SlabSpec(box=(61.5, 61.5, 246.0), ntypes=2, name=name)
    if name == "cylinder_2393":      # 24^3, liquid cylinder of radius 6 along x, N = 2,393
        return SlabSpec(box=(24.0, 24.0, 24.0), cylinder_radius=6.0, name=name)
    if name == "cylinder_299k":      # 120^3, liquid cylinder of radius 30 along x, N = 299,208
        return SlabSpec(box=(120.0, 120.0, 120.0), cylinder_radius=30.0, name=name)
    raise KeyError(name)


def _modes(seed: int, Lx: float, Ly: float, amp: float, which: int):
    """Capillary-wave mode table for one surface (empty when amp == 0)."""
    if amp == 0.0:
        e = np.zeros(0)
        return e, e, e, e
    kx, ky = np.meshgrid(np.arange(1, 5, dtype=np.float64), np.arange(1, 5, dtype=np.float64),
                         indexing="ij")
    kx, ky = kx.ravel(), ky.ravel()
    ph = 2.0 * math.pi * uniform(seed * 7919 + 101 + which, kx.size)
    a = 1.0 / np.sqrt((kx / Lx) ** 2 + (ky / Ly) ** 2)
    xs = np.linspace(0.0, Lx, 512, endpoint=False)
    ys = np.linspace(0.0, Ly, 512, endpoint=False)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    z = np.zeros_like(X)
    for m in range(kx.size):
        z += a[m] * np.cos(2.0 * math.pi * (kx[m] * X / Lx + ky[m] * Y / Ly) + ph[m])
    a = a * (amp / np.abs(z).max())
    return kx, ky, a, ph


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _surface(modes, z0, X, Y, Lx, Ly):
    kx, ky, a, ph = modes
    z = np.full_like(X, z0)
    for m in range(kx.size):
        z += a[m] * np.cos(2.0 * math.pi * (kx[m] * X / Lx + ky[m] * Y / Ly) + ph[m])
    return z


def _largest_remainder(expect: np.ndarray, total: int) -> np.ndarray:
    base = np.floor(expect).astype(np.int64)
    short = total - int(base.sum())
    if short > 0:
        order = np.argsort(-(expect - base), kind="stable")
        base[order[:short]] += 1
    elif short < 0:
        order = np.argsort(expect - base, kind="stable")
        for k in order:
            if short == 0:
                break
            if base[k] > 0:
                base[k] -= 1
                short += 1
    return base


def slab_quotas(spec: SlabSpec, nslab: int):
    """Liquid and vapor particle counts per z-slab: rho times the phase volume
    of the slab (surfaces integrated on a 512 x 512 xy grid), rounded by
    largest remainder so that the totals are exactly n_liquid and n_vapor."""
    Lx, Ly, Lz = (float(v) for v in spec.box)
    z0, z1 = spec.liquid_bounds
    lo = _modes(spec.seed, Lx, Ly, spec.wave_amp, 0)
    hi = _modes(spec.seed, Lx, Ly, spec.wave_amp, 1)
    g = 512 if spec.wave_amp > 0 else 1
    xs = (np.arange(g) + 0.5) * (Lx / g)
    ys = (np.arange(g) + 0.5) * (Ly / g)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    zl = _surface(lo, z0, X, Y, Lx, Ly)
    zh = _surface(hi, z1, X, Y, Lx, Ly)
    edges = Lz * np.arange(nslab + 1) / nslab
    area = Lx * Ly
    vliq = np.empty(nslab)
    for k in range(nslab):
        vliq[k] = area * np.clip(np.minimum(edges[k + 1], zh) - np.maximum(edges[k], zl), 0.0, None).mean()
    vslab = area * np.diff(edges)
    ql = _largest_remainder(spec.rho_l * vliq, spec.n_liquid)
    qv = _largest_remainder(spec.rho_v * (vslab - vliq), spec.n_vapor)
    return ql, qv, lo, hi


def cylinder_quotas(spec: SlabSpec, nslab: int):
    """Per-z-slab counts for the liquid cylinder: rho times the phase volume of
    the slab (the circle's chord integrated in closed form), rounded by
    largest remainder to the exact totals."""
    Lx, Ly, Lz = (float(v) for v in spec.box)
    r, zc = spec.cylinder_radius, 0.5 * Lz

    def area_below(z):  # area of the disc's part with z' < z
        t = min(max((z - zc) / r, -1.0), 1.0)
        return r * r * (t * math.sqrt(1.0 - t * t) + math.asin(t) + 0.5 * math.pi)

    edges = Lz * np.arange(nslab + 1) / nslab
    vliq = np.array([Lx * (area_below(edges[k + 1]) - area_below(edges[k])) for k in range(nslab)])
    vslab = Lx * Ly * np.diff(edges)
    ql = _largest_remainder(spec.rho_l * vliq, spec.n_liquid)
    qv = _largest_remainder(spec.rho_v * (vslab - vliq), spec.n_vapor)
    return ql, qv


def make_positions(spec: SlabSpec) -> np.ndarray:
    """RSA positions (float32, shape (N, 3), each coordinate in [0, L)); liquid
    particles first, then vapor."""
    Lx, Ly, Lz = (float(v) for v in spec.box)
    if spec.cylinder_radius > 0:
        if not 2.0 * spec.cylinder_radius < min(Ly, Lz):
            raise ValueError("the cylinder must fit in the y-z cross-section")
        nslab = max(1, int(round(Lz / 2.0)))
        ql, qv = cylinder_quotas(spec, nslab)
        pos = np.empty((int(ql.sum() + qv.sum()), 3), dtype=np.float32)
        pi64 = ctypes.POINTER(ctypes.c_int64)
        rc = _load().synth_rsa_cylinder(Lx, Ly, Lz, nslab, ql.ctypes.data_as(pi64), qv.ctypes.data_as(pi64),
                                        spec.d_min, spec.seed, spec.cylinder_radius, 0.5 * Ly, 0.5 * Lz,
                                        1000000, pos.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if rc != 0:
            raise RuntimeError(f"synth_rsa_cylinder failed ({rc}) for {spec}")
        return pos
    z0, z1 = spec.liquid_bounds
    nslab = max(1, int(round(Lz / 2.0)))
    ql, qv, lo, hi = slab_quotas(spec, nslab)
    n = int(ql.sum() + qv.sum())
    pos = np.empty((n, 3), dtype=np.float32)
    pi64 = ctypes.POINTER(ctypes.c_int64)
    rc = _load().synth_rsa_slab(Lx, Ly, Lz, nslab, ql.ctypes.data_as(pi64), qv.ctypes.data_as(pi64),
                                spec.d_min, spec.seed,
                                lo[0].size, _ptr(lo[0]), _ptr(lo[1]), _ptr(lo[2]), _ptr(lo[3]), z0,
                                hi[0].size, _ptr(hi[0]), _ptr(hi[1]), _ptr(hi[2]), _ptr(hi[3]), z1,
                                1000000, pos.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if rc != 0:
        raise RuntimeError(f"synth_rsa_slab failed ({rc}) for {spec}")
    return pos


def make_velocities(n: int, temperature: float, seed: int) -> np.ndarray:
    """Maxwell-Boltzmann velocities (m = 1), COM removed, exact kinetic temperature."""
    rng = np.random.Generator(np.random.PCG64(seed * 1000003 + 17))
    v = rng.normal(0.0, math.sqrt(temperature), size=(n, 3))
    if n > 1:
        v -= v.mean(axis=0)
        ke2 = float((v * v).sum())
        v *= math.sqrt(temperature * (3 * n - 3) / ke2)
    return v.astype(np.float32)


def make_types(n: int, ntypes: int, seed: int) -> np.ndarray:
    t = np.zeros(n, dtype=np.int32)
    if ntypes == 2:
        rng = np.random.Generator(np.random.PCG64(seed * 1000003 + 29))
        t[rng.permutation(n)[: n // 2]] = 1
    elif ntypes > 2:
        rng = np.random.Generator(np.random.PCG64(seed * 1000003 + 29))
        t[:] = rng.integers(0, ntypes, size=n)
    return t


@dataclass
class Slab:
    spec: SlabSpec
    pos: np.ndarray      # float32 (N, 3)
    vel: np.ndarray      # float32 (N, 3)
    types: np.ndarray    # int32 (N,)
    lj: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.pos.shape[0]

    @property
    def box(self):
        return tuple(float(v) for v in self.spec.box)


def _cache_path(spec: SlabSpec):
    import hashlib
    import tempfile
    if os.environ.get("DCM_SYNTH_CACHE", "1") == "0" or spec.n < 200000:
        return None
    key = repr((spec.box, spec.rho_l, spec.rho_v, spec.temperature, spec.liquid_fraction, spec.wave_amp,
                spec.ntypes, spec.d_min, spec.seed, spec.cylinder_radius, os.path.getmtime(_SRC)))
    h = hashlib.sha256(key.encode()).hexdigest()[:24]
    return os.path.join(tempfile.gettempdir(), "dcm_synth_cache", h + ".npz")


def make_slab(spec: SlabSpec) -> Slab:
    """Positions, velocities and types of one slab.  Large systems are cached
    in the system temp directory (DCM_SYNTH_CACHE=0 disables the cache)."""
    path = _cache_path(spec)
    if path and os.path.exists(path):
        try:
            z = np.load(path)
            pos, vel, types = z["pos"], z["vel"], z["types"]
        except Exception:
            path_ok = False
            pos = None
    else:
        pos = None
    if pos is None:
        pos = make_positions(spec)
        vel = make_velocities(pos.shape[0], spec.temperature, spec.seed)
        types = make_types(pos.shape[0], spec.ntypes, spec.seed)
        if path:
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                tmp = path + f".tmp{os.getpid()}.npz"
                np.savez(tmp, pos=pos, vel=vel, types=types)
                os.replace(tmp, path)
            except OSError:
                pass
    if spec.ntypes == 2:
        lj = {"eps": [1.0, 0.8], "sigma": [1.0, 1.1]}
    else:
        lj = {"eps": [1.0] * spec.ntypes, "sigma": [1.0] * spec.ntypes}
    return Slab(spec, pos, vel, types, lj)


def batch_specs(count: int = 64, n_lo: int = 2000, n_hi: int = 200000, edge: float = 1.5):
    """Independent replicas: target N log-uniform in [n_lo, n_hi], aspect
    1:1:4, rho_l ~ U[0.7, 0.85], T* ~ U[0.65, 0.85], rho_v = 0.02, seeds
    0..count-1.  The box edge is rounded to a multiple of `edge` (at least 8
    edges, so that a cutoff of 6 fits half the box); N then follows from the
    densities."""
    out = []
    for s in range(count):
        u = uniform(100000 + s, 3)
        n_target = math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))
        rho_l = 0.7 + 0.15 * u[1]
        temp = 0.65 + 0.2 * u[2]
        # N = L^2 * 4L * (rho_l/3 + 2 rho_v/3)
        L = (n_target / (4.0 * (rho_l + 2.0 * 0.02) / 3.0)) ** (1.0 / 3.0)
        L = edge * max(8, int(round(L / edge)))
        out.append(SlabSpec(box=(L, L, 4.0 * L), rho_l=rho_l, temperature=temp, seed=s, name=f"replica_{s}"))
    return out
