"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: closed
forms, brute force, library routines that solve a special case, invariances,
values the paper prints (tests/golden/), or convergence orders.  A plausible
slip in the oracle (dropped term, wrong sign or index, swapped operand) breaks
at least one of these.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- LJ pair ---
def two_particles(r, rc_i=6.0, rc_j=6.0, box=(24.0, 24.0, 24.0), shift=False):
    pos = np.array([[5.0, 7.0, 9.0], [5.0 + r, 7.0, 9.0]])
    return O.forces_brute(pos, np.array([rc_i, rc_j]), box, shift=shift)


def test_lj_closed_forms():
    # U(sigma) = 0, |F|(sigma) = 24 eps/sigma, minimum U = -eps at 2^(1/6) sigma with F = 0
    r = two_particles(1.0)
    assert abs(r.E) < 1e-13
    assert r.F[0, 0] == pytest.approx(-24.0, rel=1e-14)        # pushed away from j (j at +x)
    assert r.F[1, 0] == pytest.approx(24.0, rel=1e-14)
    rmin = 2.0 ** (1.0 / 6.0)
    r = two_particles(rmin)
    assert r.E == pytest.approx(-1.0, rel=1e-13)
    assert abs(r.F[0, 0]) < 1e-12
    # long range: U r^6 -> -4 eps sigma^6, attractive force
    r = two_particles(5.0)
    assert r.E * 5.0 ** 6 == pytest.approx(-4.0, rel=1e-3)
    assert r.F[0, 0] > 0.0
    # virial of one pair: W = r . F_ij = r |F|; at r = sigma: 24
    r = two_particles(1.0)
    assert r.W == pytest.approx(24.0, rel=1e-14)


def test_lj_mixing_lorentz_berthelot():
    # eps_ab = sqrt(eps_a eps_b), sigma_ab = (sigma_a + sigma_b)/2: minimum of the
    # mixed pair sits at 2^(1/6) sigma_ab with depth eps_ab.
    eps, sig = (1.0, 0.8), (1.0, 1.1)
    s01 = 1.05
    pos = np.array([[3.0, 3.0, 3.0], [3.0 + 2 ** (1 / 6) * s01, 3.0, 3.0]])
    r = O.forces_brute(pos, np.array([6.0, 6.0]), (20.0,) * 3, types=np.array([0, 1]), eps=eps, sigma=sig)
    assert r.E == pytest.approx(-math.sqrt(0.8), rel=1e-13)
    assert abs(r.F[0, 0]) < 1e-12


def test_strict_cutoff_comparison():
    # j is included iff |r_ij| < rc_i (strict): r = 3 exactly
    r = two_particles(3.0, rc_i=3.0, rc_j=3.0)
    assert r.npairs == 0 and r.E == 0.0
    r = two_particles(3.0, rc_i=math.nextafter(3.0, 4.0), rc_j=3.0)
    assert r.npairs == 1
    assert r.F[0, 0] != 0.0 and r.F[1, 0] == 0.0


def test_asymmetric_cutoffs_no_newton3():
    # Section 2.4: i influenced by j does not imply j influenced by i.
    r = two_particles(4.0, rc_i=3.0, rc_j=6.0)
    both = two_particles(4.0, rc_i=6.0, rc_j=6.0)
    assert r.npairs == 1
    assert np.all(r.F[0] == 0.0)
    assert np.array_equal(r.F[1], both.F[1])
    assert r.E == pytest.approx(0.5 * both.E, rel=1e-15)


def test_shifted_energy_zero_at_cutoff():
    # shifted pair energy U(r) - U(rc) vanishes as r -> rc from below; force unchanged
    rc = 3.0
    r = two_particles(math.nextafter(rc, 0.0), rc_i=rc, rc_j=rc, shift=True)
    assert abs(r.E) < 1e-12
    a = two_particles(2.0, rc_i=rc, rc_j=rc, shift=True)
    b = two_particles(2.0, rc_i=rc, rc_j=rc, shift=False)
    assert np.array_equal(a.F, b.F)
    u2, _ = O.lj_pair(2.0)
    uc, _ = O.lj_pair(rc)
    assert a.E - b.E == pytest.approx(-uc, rel=1e-12)


# ------------------------------------------------------- forces: systems ---
def _classical_cutoff_lj(pos, box, rc):
    """Eq. 3 written independently: symmetric pair loop i < j with Newton's
    third law, minimum image by rounding, numpy vectorised per i."""
    pos = np.asarray(pos, np.float64)
    box = np.asarray(box, np.float64)
    n = len(pos)
    F = np.zeros((n, 3))
    E = 0.0
    W = 0.0
    for i in range(n - 1):
        d = pos[i] - pos[i + 1:]
        d -= box * np.round(d / box)
        r2 = (d * d).sum(1)
        m = r2 < rc * rc
        inv6 = 1.0 / r2[m] ** 3
        fs = 24.0 * (2.0 * inv6 * inv6 - inv6) / r2[m]
        fij = fs[:, None] * d[m]
        F[i] += fij.sum(0)
        F[i + 1:][m] -= fij
        E += (4.0 * (inv6 * inv6 - inv6)).sum()
        W += (fs * r2[m]).sum()
    return F, E, W


def test_uniform_cutoff_is_classical_lj(slab_1935):
    # rc_min = rc_max: DCM reduces to the static cutoff method (Eq. 3)
    pos, box = slab_1935.pos.astype(np.float64), slab_1935.box
    rc = 3.0
    got = O.forces_cells(pos, rc, box, 1.5)
    F, E, W = _classical_cutoff_lj(pos, box, rc)
    scale = np.abs(F).max()
    assert np.abs(got.F - F).max() < 1e-12 * scale
    assert got.E == pytest.approx(E, rel=1e-12)
    assert got.W == pytest.approx(W, rel=1e-12)
    # Newton's third law holds in the uniform case: zero net force
    assert np.abs(got.F.sum(0)).max() < 1e-12 * np.abs(got.F).sum()


def test_uniform_force_is_minus_energy_gradient(slab_1935):
    pos, box = slab_1935.pos.astype(np.float64), np.array(slab_1935.box)
    rc = 3.0
    base = O.forces_brute(pos, rc, box, shift=True)
    rng = np.random.default_rng(5)
    checked = 0
    for i in rng.permutation(len(pos))[:40]:
        d = pos[i] - pos
        d -= box * np.round(d / box)
        r = np.sqrt((d * d).sum(1))
        r[i] = np.inf
        if np.min(np.abs(r - rc)) < 1e-3:
            continue  # a pair would cross the cutoff under the perturbation
        for k in range(3):
            hstep = 1e-6
            pp, pm = pos.copy(), pos.copy()
            pp[i, k] += hstep
            pm[i, k] -= hstep
            ep = O.forces_brute(pp, rc, box, shift=True).E
            em = O.forces_brute(pm, rc, box, shift=True).E
            fd = -(ep - em) / (2 * hstep)
            assert fd == pytest.approx(base.F[i, k], rel=2e-6, abs=2e-5)
        checked += 1
        if checked == 5:
            break
    assert checked == 5


def test_brute_force_equals_cells(slab_1935):
    pos, box = slab_1935.pos.astype(np.float64), slab_1935.box
    rng = np.random.default_rng(1)
    rc = rng.uniform(3.0, 6.0, len(pos))
    a = O.forces_brute(pos, rc, box)
    for l in (1.5, 3.0, 0.75):
        b = O.forces_cells(pos, rc, box, l, nthreads=2)
        assert a.npairs == b.npairs
        assert np.abs(a.F - b.F).max() < 1e-12 * np.abs(a.F).max()
        assert np.abs(a.e - b.e).max() < 1e-12 * np.abs(a.e).max()
        assert b.E == pytest.approx(a.E, rel=1e-12)
        assert b.W == pytest.approx(a.W, rel=1e-12)


@pytest.mark.parametrize("l", [1.5, (0.5, 1.5, 1.5)])
def test_forces_subset_equals_brute_rows(slab_1935, l):
    # the sampled form used at full sizes: its rows and per-particle sums
    # against the O(N^2) pair loop, two types and the shifted energy
    pos, box = slab_1935.pos.astype(np.float64), slab_1935.box
    rng = np.random.default_rng(11)
    n = len(pos)
    rc = rng.uniform(3.0, 6.0, n)
    types = (np.arange(n) % 2).astype(np.int32)
    kw = dict(types=types, eps=(1.0, 0.8), sigma=(1.0, 1.1), shift=True)
    a = O.forces_brute(pos, rc, box, **kw)
    every = np.arange(n)
    F, e, w, npairs = O.forces_subset(pos, rc, box, l, every, **kw)
    assert np.abs(F - a.F).max() < 1e-12 * np.abs(a.F).max()
    assert np.abs(e - a.e).max() < 1e-12 * np.abs(a.e).max()
    assert int(npairs.sum()) == a.npairs
    assert w.sum() == pytest.approx(a.W, rel=1e-12)
    idx = rng.choice(n, 37, replace=False)
    F, e, w, npairs = O.forces_subset(pos, rc, box, l, idx, **kw)
    assert np.abs(F - a.F[idx]).max() < 1e-12 * np.abs(a.F).max()
    assert np.abs(e - a.e[idx]).max() < 1e-12 * np.abs(a.e).max()
    # per-particle pair count by direct minimum-image distances
    d = pos[idx, None, :] - pos[None, :, :]
    d -= np.asarray(box) * np.round(d / np.asarray(box))
    r2 = (d * d).sum(-1)
    r2[np.arange(37), idx] = np.inf
    assert np.array_equal(npairs, (r2 < rc[idx, None] ** 2).sum(1))


def test_dcm_force_is_per_particle_uniform(slab_1935):
    # F_i under DCM equals the uniform-cutoff force at r_c = rc_i, evaluated at i
    pos, box = slab_1935.pos.astype(np.float64), slab_1935.box
    rng = np.random.default_rng(2)
    rc = rng.choice([3.0, 4.5, 6.0], len(pos))
    dcm = O.forces_brute(pos, rc, box)
    for val in (3.0, 4.5, 6.0):
        uni = O.forces_brute(pos, val, box)
        m = rc == val
        assert np.array_equal(dcm.F[m], uni.F[m])
        assert np.array_equal(dcm.e[m], uni.e[m])


def test_translation_and_permutation_invariance(slab_1935):
    pos, box = slab_1935.pos.astype(np.float64), np.array(slab_1935.box)
    rng = np.random.default_rng(3)
    rc = rng.uniform(3.0, 6.0, len(pos))
    a = O.forces_cells(pos, rc, box, 1.5)
    moved = np.mod(pos + np.array([3.25, -7.5, 11.0]), box)
    b = O.forces_cells(moved, rc, box, 1.5)
    assert a.npairs == b.npairs
    assert np.abs(a.F - b.F).max() < 1e-9 * np.abs(a.F).max()
    assert b.E == pytest.approx(a.E, rel=1e-11)
    perm = rng.permutation(len(pos))
    c = O.forces_cells(pos[perm], rc[perm], box, 1.5)
    # the j order inside a cell follows the input order, so only rounding may differ
    assert np.abs(c.F - a.F[perm]).max() < 1e-12 * np.abs(a.F).max()
    assert c.npairs == a.npairs
    assert c.E == pytest.approx(a.E, rel=1e-13)


def test_dcm_net_force_nonzero_reported(slab_1935):
    # with per-particle cutoffs Newton's third law does not hold (Section 2.4)
    pos, box = slab_1935.pos.astype(np.float64), slab_1935.box
    p = O.Params(box=box)
    rc = O.assign_cutoffs(pos, p)["rc"]
    r = O.forces_cells(pos, rc, box, 1.5)
    assert np.abs(r.F.sum(0)).max() > 1e-6


# --------------------------------------------------------------- binning ---
def test_binning_properties(slab_1935):
    pos, box = slab_1935.pos.astype(np.float64), np.array(slab_1935.box)
    for l in (1.5, 1.0, 0.75, (0.75, 1.5, 1.5), (0.5, 1.5, 1.5)):
        cell, count, start, perm = O.bin_particles(pos, box, l)
        nc = O.grid_dims(box, l)
        l = np.broadcast_to(np.asarray(l, np.float64), (3,))
        assert count.sum() == len(pos)
        assert start[0] == 0 and start[-1] == len(pos)
        assert np.array_equal(np.diff(start), count)
        cx = cell % nc[0]
        cy = (cell // nc[0]) % nc[1]
        cz = cell // (nc[0] * nc[1])
        c3 = np.stack([cx, cy, cz], 1)
        assert np.all(c3 * l <= pos) and np.all(pos < (c3 + 1) * l)
        # stable order: numpy's stable sort by cell
        assert np.array_equal(perm, np.argsort(cell, kind="stable"))


def test_cell_coord_exact_floor_at_boundaries():
    l = 1.5
    for k in (1, 2, 7, 100, 639):
        x = np.float32(k * l)
        assert O.cell_coord(float(x), l, 1000) == k
        below = np.nextafter(np.float32(k * l), np.float32(0))
        assert O.cell_coord(float(below), l, 1000) == k - 1
    assert O.cell_coord(0.0, l, 8) == 0
    assert O.cell_coord(12.0, l, 8) == 7   # clamped


# ------------------------------------------------------------- interface ---
def test_two_means_matches_exhaustive_split():
    # 2-means on bimodal data reaches the split minimising within-class SSE
    rng = np.random.default_rng(4)
    g = np.concatenate([rng.poisson(8, 300), rng.poisson(300, 200)]).astype(np.int32)
    T = O.two_means(g)
    best, bestT = None, None
    for t in range(int(g.min()) + 1, int(g.max()) + 1):
        a, b = g[g < t], g[g >= t]
        if len(a) == 0 or len(b) == 0:
            continue
        sse = ((a - a.mean()) ** 2).sum() + ((b - b.mean()) ** 2).sum()
        if best is None or sse < best - 1e-9:
            best, bestT = sse, t
    assert np.array_equal(g >= T, g >= bestT)
    # hand example: {1,1,1,9,9,9} -> means 1 and 9, midpoint 5, s = g > 5
    assert O.two_means(np.array([1, 1, 1, 9, 9, 9], np.int32)) == 6
    # one phase only: no interface
    assert O.two_means(np.full(10, 7, np.int32)) == 8


def test_interface_hand_grids():
    nh = np.array([6, 5, 8])
    n = int(np.prod(nh))
    # all liquid: uniform counts -> single phase -> no interface
    g, T, s, iface = O.detect_interface(np.full(n, 3, np.int32), nh, 1)
    assert iface.sum() == 0
    # half-space in z: counts 10 for z >= 4, 0 below -> two interface planes
    # (z = 4 facing z = 3, and z = 7 facing z = 0 through the periodic wrap)
    c = np.zeros((nh[2], nh[1], nh[0]), np.int32)
    c[4:] = 10
    g, T, s, iface = O.detect_interface(c.ravel(), nh, 0)
    I = iface.reshape(nh[2], nh[1], nh[0])
    assert I[4].all() and I[7].all() and I.sum() == 2 * nh[0] * nh[1]
    S = s.reshape(I.shape)
    assert S[4:].all() and not S[:4].any()
    # smoothing is the plain box sum: w = 1 on a single particle gives a 3x3x3 block of ones
    c = np.zeros(n, np.int32)
    c[0] = 1
    g = O.smooth(c, nh, 1).reshape(nh[2], nh[1], nh[0])
    assert g.sum() == 27 and g[0, 0, 0] == 1 and g[-1, -1, -1] == 1 and g[1, 1, 1] == 1 and g[2, 2, 2] == 0


# ------------------------------------------------------------ distances ---
def test_cfsm_planar_interface_exact():
    nh = np.array([4, 4, 20])
    s = np.zeros((20, 4, 4), np.uint8)
    s[5:17] = 1
    iface = np.zeros_like(s)
    iface[5] = 1
    iface[16] = 1
    h, rg = 1.5, 6.0
    D, it = O.cfsm(s.ravel(), iface.ravel(), nh, h, rg)
    D = D.reshape(s.shape)
    inf = np.inf
    expect = [0, 0, 0, 0, 0, 0, 1.5, 3.0, 4.5, 6.0, inf, inf, 6.0, 4.5, 3.0, 1.5, 0, 0, 0, 0]
    for z, e in enumerate(expect):
        assert np.all(D[z] == e), (z, D[z, 0, 0], e)
    assert it <= rg / h + 2


def test_cfsm_point_source_godunov_values():
    # one seed box in a high-density volume: the published Godunov update gives
    # h on faces, (1 + sqrt(2)/2) h on edge diagonals, and that + h/sqrt(3) on corners
    nh = np.array([9, 9, 9])
    s = np.ones(729, np.uint8)
    iface = np.zeros(729, np.uint8)
    c = 4 + 9 * (4 + 9 * 4)
    iface[c] = 1
    h = 1.5
    D, _ = O.cfsm(s, iface, nh, h, 100.0)
    D = D.reshape(9, 9, 9)
    e2 = (1 + math.sqrt(2) / 2) * h
    assert D[4, 4, 5] == pytest.approx(h, rel=1e-15)
    assert D[4, 5, 5] == pytest.approx(e2, rel=1e-15)
    assert D[5, 5, 5] == pytest.approx(e2 + h / math.sqrt(3), rel=1e-14)


def _random_blob(nh, rng):
    s = np.ones(int(np.prod(nh)), np.uint8)
    iface = (rng.random(s.size) < 0.003).astype(np.uint8)
    s[rng.random(s.size) < 0.002] = 0
    return s, iface


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cfsm_vs_brute_euclid_and_orderings(seed):
    rng = np.random.default_rng(seed)
    nh = np.array([14, 12, 16])
    s, iface = _random_blob(nh, rng)
    h, rg = 1.5, 7.5
    Dq, itq = O.cfsm(s, iface, nh, h, rg)
    Dj, itj = O.distance_jacobi(s, iface, nh, h, rg)
    Ds, its = O.distance_sweep8(s, iface, nh, h, rg)
    fin = np.isfinite(Dj)
    # order independence (the paper: same result as Zhao's sweeps within r_grid)
    assert np.array_equal(np.isfinite(Dq), fin) and np.array_equal(np.isfinite(Ds), fin)
    assert np.abs(Dq[fin] - Dj[fin]).max() <= 1e-12
    assert np.abs(Ds[fin] - Dj[fin]).max() <= 1e-12
    # Jacobi sweeps grow with the longest dependency chain (about the L1 length
    # of r_grid / h); the queue version updates in place, so last-ulp
    # improvements can ripple for a few extra passes
    assert itj <= 3 * rg / h + 2
    assert itq <= 5 * rg / h + 2
    # brute-force Euclidean distance between box centres and the nearest seed (periodic)
    seeds = np.flatnonzero((s == 0) | (iface == 1))
    idx = np.arange(s.size)
    X = np.stack([idx % nh[0], (idx // nh[0]) % nh[1], idx // (nh[0] * nh[1])], 1).astype(float)
    S = X[seeds]
    d = X[:, None, :] - S[None, :, :]
    d -= nh * np.round(d / nh)
    de = h * np.sqrt((d * d).sum(-1)).min(1)
    # the first-order upwind solution undershoots by less than half a box and
    # overshoots by at most about a third of the distance (point sources seen
    # along lattice diagonals; measured: -0.42 h and +0.32 d on these grids)
    err = Dj[fin] - de[fin]
    assert np.all(err >= -0.5 * h)
    assert np.all(err <= 0.35 * np.maximum(de[fin], h))
    # boxes left at +inf lie beyond r_grid up to the same overshoot
    assert (~fin).sum() > 0
    assert np.all(de[~fin] * 1.35 > rg)


def test_cfsm_iteration_cap_reports_failure():
    nh = np.array([4, 4, 40])
    s = np.ones(640, np.uint8)
    iface = np.zeros(640, np.uint8)
    iface[:16] = 1
    D, it = O.cfsm(s, iface, nh, 1.0, 100.0, iter_max=3)
    assert it == -1


# --------------------------------------------------------------- cutoffs ---
def test_cutoff_rule_endpoints_and_monotone():
    assert O.cutoff_rule(0.0, 3.0, 6.0, 3.0) == 6.0
    assert O.cutoff_rule(3.0, 3.0, 6.0, 3.0) == 3.0
    assert O.cutoff_rule(10.0, 3.0, 6.0, 3.0) == 3.0
    vals = [O.cutoff_rule(d, 3.0, 6.0, 3.0) for d in np.linspace(0, 5, 101)]
    assert all(a >= b for a, b in zip(vals, vals[1:]))


def test_trilinear_reproduces_linear_fields():
    # trilinear interpolation is exact for fields linear in x, y, z
    nh = np.array([10, 10, 10])
    h = 1.5
    idx = np.arange(1000)
    X = np.stack([idx % 10, (idx // 10) % 10, idx // 100], 1)
    D = 0.2 * (X[:, 0] + 0.5) * h + 0.1 * (X[:, 1] + 0.5) * h + 0.05 * (X[:, 2] + 0.5) * h
    rng = np.random.default_rng(6)
    p = rng.uniform(1.0, 13.0, size=(50, 3))   # stay away from the periodic seam
    delta, _ = O.cutoffs(p, D, nh, h, 1e9, 3.0, 6.0, 3.0)
    assert np.abs(delta - (0.2 * p[:, 0] + 0.1 * p[:, 1] + 0.05 * p[:, 2])).max() < 1e-12


def test_trilinear_periodic_seam_hand_values():
    """Section 2.2's interpolation between box centres (k + 1/2) h, periodic:
    within h/2 of a face a particle sits between the centre of the last box
    (its image at -h/2, or at L - h/2) and that of box 0 (at h/2, or its image
    at L + h/2).  The field differs on the two sides of every seam, so a wrap
    to the wrong box or a missing wrap changes the value.  Expected values are
    written out by hand for these positions."""
    h = 1.5
    nh = np.array([4, 5, 6])
    L = nh * h
    # every box 5.0 except the boxes at both ends of each axis
    D = np.full(int(np.prod(nh)), 5.0)

    def box(x, y, z):
        return x + nh[0] * (y + nh[1] * z)

    # a y-z interior line of boxes (y = 2, z = 3) with distinct end values along x
    D[box(3, 2, 3)] = 1.0   # last box along x
    D[box(0, 2, 3)] = 2.5   # first box along x
    D[box(1, 2, 3)] = 0.5
    D[box(2, 2, 3)] = 4.0
    yc, zc = (2 + 0.5) * h, (3 + 0.5) * h   # box centres: no weight on y, z neighbours
    pts = np.array([
        [0.0, yc, zc],              # halfway between box 3's image and box 0
        [0.25 * h, yc, zc],         # 3/4 of the way to box 0
        [L[0] - 0.25 * h, yc, zc],  # 1/4 of the way from box 3 to box 0's image
        [L[0] - 1e-9, yc, zc],      # just below L: almost halfway
        [0.5 * h, yc, zc],          # box 0's centre exactly
        [L[0] - 0.5 * h, yc, zc],   # box 3's centre exactly
    ])
    want = np.array([
        0.5 * 1.0 + 0.5 * 2.5,
        0.25 * 1.0 + 0.75 * 2.5,
        0.75 * 1.0 + 0.25 * 2.5,
        0.5 * 1.0 + 0.5 * 2.5,
        2.5,
        1.0,
    ])
    delta, _ = O.cutoffs(pts, D, nh, h, 1e9, 3.0, 6.0, 3.0)
    assert np.allclose(delta, want, rtol=0, atol=1e-8), (delta, want)

    # the same along y and z: a line of boxes along y (x = 1, z = 2) and along z (x = 2, y = 1)
    D2 = np.full(int(np.prod(nh)), 5.0)
    D2[box(1, 4, 2)], D2[box(1, 0, 2)] = 0.25, 3.25    # y: last box, first box
    D2[box(2, 1, 5)], D2[box(2, 1, 0)] = 2.0, 0.75     # z: last box, first box
    xc1, zc2 = 1.5 * h, 2.5 * h
    pts = np.array([
        [xc1, 0.0, zc2],                     # y seam: halfway
        [xc1, L[1] - 0.25 * h, zc2],         # y seam: 1/4 past the last centre
        [2.5 * h, 1.5 * h, 0.0],             # z seam: halfway
        [2.5 * h, 1.5 * h, 0.25 * h],        # z seam: 3/4 of the way to box 0
    ])
    want = np.array([
        0.5 * 0.25 + 0.5 * 3.25,
        0.75 * 0.25 + 0.25 * 3.25,
        0.5 * 2.0 + 0.5 * 0.75,
        0.25 * 2.0 + 0.75 * 0.75,
    ])
    delta, _ = O.cutoffs(pts, D2, nh, h, 1e9, 3.0, 6.0, 3.0)
    assert np.allclose(delta, want, rtol=0, atol=1e-8), (delta, want)

    # the corner (0, 0, 0): the mean of the eight boxes at the ends of all
    # three axes, with values that differ box by box
    D3 = np.full(int(np.prod(nh)), 5.0)
    corners = {}
    v = 0.125
    for cz in (nh[2] - 1, 0):
        for cy in (nh[1] - 1, 0):
            for cx in (nh[0] - 1, 0):
                D3[box(cx, cy, cz)] = v
                corners[(cx, cy, cz)] = v
                v += 0.375
    delta, _ = O.cutoffs(np.zeros((1, 3)), D3, nh, h, 1e9, 3.0, 6.0, 3.0)
    assert abs(delta[0] - sum(corners.values()) / 8.0) < 1e-12

    # values above r_grid are capped before they are interpolated
    delta, _ = O.cutoffs(np.array([[0.0, yc, zc]]), D, nh, h, 2.0, 3.0, 6.0, 3.0)
    assert abs(delta[0] - (0.5 * 1.0 + 0.5 * 2.0)) < 1e-12


def test_slab_cutoffs(slab_1935):
    pos = slab_1935.pos.astype(np.float64)
    p = O.Params(box=slab_1935.box)
    a = O.assign_cutoffs(pos, p)
    z = pos[:, 2]
    assert np.all(a["rc"] >= 3.0) and np.all(a["rc"] <= 6.0)
    # vapor far from the slab: largest cutoff; liquid centre: smallest
    assert np.all(a["rc"][(z < 10) | (z > 38)] == 6.0)
    assert np.all(a["rc"][(z > 22) & (z < 26)] == 3.0)
    assert a["iface"].sum() == 2 * 8 * 8


# ---------------------------------------------------- paper's arithmetic ---
def test_paper_volume_ratio_golden():
    gold = json.load(open(os.path.join(GOLDEN, "paper_values.json")))
    v = gold["stencil_volume_ratio"]
    rc_max = 1.0
    rc_min = v["rc_min_over_rc_max"] * rc_max
    rs = v["skin_over_rc_max"] * rc_max
    ratio = (4.0 / 3.0 * math.pi * rc_min ** 3) / (3.0 * (rc_max + rs)) ** 3
    assert ratio == pytest.approx(v["value"], abs=v["abs_tol"])


# ------------------------------------------------------------------ NVE ---
def test_velocity_verlet_second_order(slab_1935):
    p = O.Params(box=slab_1935.box, rc_min=3.0, rc_max=3.0, shift=True)
    errs = []
    for dt, ns in ((0.004, 25), (0.002, 50)):
        st = O.init_state(slab_1935.pos, slab_1935.vel, p)
        e0 = st.E + O.kinetic(st.vel)
        for _ in range(ns):
            st = O.step(st, dt, p)
        errs.append(abs(st.E + O.kinetic(st.vel) - e0) / abs(e0))
    assert 3.0 < errs[0] / errs[1] < 5.5


def test_kick_drift_wrap():
    pos = np.array([[0.01, 5.0, 11.99]])
    vel = np.array([[-4.0, 0.0, 4.0]])
    out = O.drift(pos, vel, 0.005, (12.0, 12.0, 12.0))
    assert out[0, 0] == pytest.approx(11.99, abs=1e-12)
    assert out[0, 2] == pytest.approx(0.01, abs=1e-12)
    v = O.kick(vel, np.array([[2.0, 2.0, 2.0]]), 0.5)
    assert np.array_equal(v, [[-3.0, 1.0, 5.0]])


# ------------------------------------------------------------ bubble filter
def _uf_components(s, nh):
    """Independent check: union-find over face links (periodic), pure Python."""
    nx, ny, nz = (int(v) for v in nh)
    parent = list(range(s.size))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                b = x + nx * (y + ny * z)
                for n in (((x + 1) % nx) + nx * (y + ny * z), x + nx * (((y + 1) % ny) + ny * z),
                          x + nx * (y + ny * ((z + 1) % nz))):
                    if s[n] == s[b]:
                        ra, rb = find(b), find(n)
                        if ra != rb:
                            parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(b) for b in range(s.size)])
    return roots, np.bincount(roots, minlength=s.size)


def test_bubble_filter_hand_built():
    nh = np.array([10, 10, 10])
    s = np.zeros((10, 10, 10), np.uint8)        # [z, y, x]
    s[2:8] = 1                                  # liquid slab
    s[4:6, 4:6, 4:6] = 0                        # vapor bubble of 8 boxes
    s[3:6, 1:4, 7:10] = 0                       # vapor bubble of 27 boxes
    s[0, 5, 5] = 1                              # liquid droplet of 1 box in vapor
    out, k = O.remove_small_components(s.ravel(), nh, 10)
    exp = np.zeros_like(s)
    exp[2:8] = 1
    exp[3:6, 1:4, 7:10] = 0                     # the large bubble stays
    assert k == 2 and np.array_equal(out.reshape(s.shape), exp)
    # interface of the filtered volume: the slab faces and the large bubble's skin
    iface = O.interface(out, nh).reshape(s.shape)
    assert iface[2].all() and iface[7].all() and iface[6, 2, 8] == 1 and iface[4, 4, 4] == 0


def test_bubble_filter_periodic_and_strict():
    nh = np.array([8, 6, 6])
    s = np.ones((6, 6, 8), np.uint8)
    s[2:4, 2, 0] = 0
    s[2:4, 2, 7] = 0                            # one 4-box bubble across the x boundary
    out4, k4 = O.remove_small_components(s.ravel(), nh, 4)
    out5, k5 = O.remove_small_components(s.ravel(), nh, 5)
    assert k4 == 0 and np.array_equal(out4, s.ravel())     # size 4 is not < 4
    assert k5 == 1 and out5.all()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bubble_filter_matches_union_find(seed):
    rng = np.random.default_rng(seed)
    nh = np.array([7, 6, 5])
    s = (rng.random(210) < 0.55).astype(np.uint8)
    roots, size = _uf_components(s, nh)
    for m in (2, 4, 9):
        out, k = O.remove_small_components(s, nh, m)
        small = size[roots] < m
        assert np.array_equal(out, np.where(small, 1 - s, s))
        assert k == len(set(roots[small].tolist()))
    # translation invariance
    sh = np.roll(s.reshape(5, 6, 7), (1, 2, 3), axis=(0, 1, 2)).ravel()
    o1, _ = O.remove_small_components(s, nh, 4)
    o2, _ = O.remove_small_components(sh, nh, 4)
    assert np.array_equal(np.roll(o1.reshape(5, 6, 7), (1, 2, 3), axis=(0, 1, 2)).ravel(), o2)
