"""The curved-interface workload (a liquid cylinder in vapor, Fig. 5b) on the
oracle, pinned to its geometry: the generator's phases and counts, the
detected interface on the cylinder's surface, CFSM distances against brute
force Euclidean distances, and cutoffs that fall toward the axis.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1701_05242_gb300 import synth


@pytest.fixture(scope="module")
def cyl():
    return synth.make_slab(synth.named("cylinder_2393"))


def axis_distance(p, box):
    return np.sqrt((p[:, 1] - 0.5 * box[1]) ** 2 + (p[:, 2] - 0.5 * box[2]) ** 2)


def box_centres(nh, h):
    idx = np.arange(int(np.prod(nh)))
    k = np.stack([idx % nh[0], (idx // nh[0]) % nh[1], idx // (nh[0] * nh[1])], 1)
    return (k + 0.5) * h, k


def test_generator_phases_and_counts(cyl):
    spec = cyl.spec
    R, L = spec.cylinder_radius, spec.box
    assert spec.n_liquid == math.floor(0.8 * math.pi * R * R * L[0] + 0.5)
    assert spec.n_vapor == math.floor(0.02 * (L[0] * L[1] * L[2] - math.pi * R * R * L[0]) + 0.5)
    r = axis_distance(cyl.pos.astype(np.float64), L)
    assert (r[:spec.n_liquid] < R).all() and (r[spec.n_liquid:] >= R).all()
    # RSA minimum distance 0.85 (periodic), checked exhaustively
    p = cyl.pos.astype(np.float64)
    for i in range(0, len(p), 7):
        d = p - p[i]
        d -= np.array(L) * np.round(d / np.array(L))
        r2 = (d * d).sum(1)
        r2[i] = 1e9
        assert r2.min() >= 0.85 ** 2 * (1 - 1e-6)


def test_interface_lies_on_the_cylinder_surface(cyl):
    nh = O.grid_dims(cyl.box, 1.5)
    _, count, _, _ = O.bin_particles(cyl.pos, cyl.box, 1.5)
    g, T, s, iface = O.detect_interface(count, nh, 2)
    X, k = box_centres(nh, 1.5)
    r = axis_distance(X, cyl.box)
    R = cyl.spec.cylinder_radius
    assert iface.sum() > 0
    assert np.abs(r[iface == 1] - R).max() <= 1.5            # within one box of the surface
    assert (s[r < R - 3.0] == 1).all() and (s[r > R + 3.0] == 0).all()
    # the interface is a closed ring in every x-plane of boxes
    for x in range(nh[0]):
        assert iface[k[:, 0] == x].sum() > 0


def test_cfsm_on_curved_front_vs_brute_force(cyl):
    nh = O.grid_dims(cyl.box, 1.5)
    _, count, _, _ = O.bin_particles(cyl.pos, cyl.box, 1.5)
    g, T, s, iface = O.detect_interface(count, nh, 2)
    h, rg = 1.5, 6.0
    D, _ = O.cfsm(s, iface, nh, h, rg)
    Dj, _ = O.distance_jacobi(s, iface, nh, h, rg)
    fin = np.isfinite(D)
    assert np.array_equal(fin, np.isfinite(Dj)) and np.abs(D[fin] - Dj[fin]).max() <= 1e-12
    seeds = np.flatnonzero((s == 0) | (iface == 1))
    _, k = box_centres(nh, 1.0)
    d = k[:, None, :].astype(float) - k[seeds][None, :, :]
    d -= nh * np.round(d / nh)
    de = h * np.sqrt((d * d).sum(-1)).min(1)
    # the first-order upwind solution against box-centre seeds: the same
    # bounds as on the random fronts (undershoot < h/2, overshoot <= 0.35 d)
    err = D[fin] - de[fin]
    assert np.all(err >= -0.5 * h)
    assert np.all(err <= 0.35 * np.maximum(de[fin], h))
    # deepest boxes: the distance grows toward the axis
    X, _ = box_centres(nh, h)
    r = axis_distance(X, cyl.box)
    assert D[r < 1.5].min() > D[(r > 3.0) & (r < 4.5)].max() - 1e-12


def test_cutoffs_fall_toward_the_axis(cyl):
    a = O.assign_cutoffs(cyl.pos, O.Params(box=cyl.box))
    r = axis_distance(cyl.pos.astype(np.float64), cyl.box)
    rc = a["rc"]
    assert (rc[r > cyl.spec.cylinder_radius + 3.0] == 6.0).all()   # vapor beyond the band: rc_max
    assert (rc[r < 1.0] < 6.0).all()                               # near the axis: reduced
    assert rc[r < 1.0].mean() < rc[(r > 4.0) & (r < 5.0)].mean()
    assert ((rc >= 3.0) & (rc <= 6.0)).all()
