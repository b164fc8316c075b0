"""Pins of the oracle's regularised two-phase Mumford-Shah segmentation
(Section 2.1; the functional of refs. [1, 18] with the reading stated in
oracle/dcm_oracle.c): closed-form thresholds of the length term, the special
case nu = 0 that reduces to 2-means, brute-force minima on tiny periodic
grids, and invariances."""
import itertools

import numpy as np
import pytest

import oracle as O


def test_isolated_box_closed_form():
    """An empty box inside a liquid of count 4 (vapor of count 0 elsewhere):
    filling it costs (0 - 4)^2 = 16 of data and saves its six faces, so it is
    filled exactly when 6 nu > 16."""
    nh = np.array([6, 6, 6])
    g = np.zeros(216, np.int32)
    z = np.arange(216) // 36
    g[z >= 3] = 4
    hole = 2 + 6 * (2 + 6 * 4)
    g[hole] = 0
    s0 = (g >= 2).astype(np.uint8)
    for nu, filled in ((2.5, 0), (2.6, 0), (2.7, 1), (3.5, 1)):
        s, u, c, k = O.ms_segment(g, nh, s0, nu, 400, 5)
        assert s[hole] == filled, nu
        # every other box keeps its phase: the planar interfaces are minimal
        rest = np.arange(216) != hole
        assert np.array_equal(s[rest], s0[rest])


def test_nu_zero_is_two_means_of_the_counts():
    """Without the length term the minimiser for fixed phase values is the
    threshold at their midpoint, and the outer loop is Lloyd's 2-means: the
    result is the integer 2-means threshold of the (unsmoothed) counts."""
    rng = np.random.default_rng(3)
    nh = np.array([8, 8, 16])
    z = np.arange(int(np.prod(nh))) // 64
    g = np.where((z >= 4) & (z < 12), rng.poisson(9.0, z.size), rng.poisson(0.7, z.size)).astype(np.int32)
    T = O.two_means(g)
    s0 = (g >= 5).astype(np.uint8)
    s, u, (c0, c1), k = O.ms_segment(g, nh, s0, 0.0, 50, 64)
    tie = np.abs(g - 0.5 * (c0 + c1)) < 1e-12
    assert np.array_equal(s[~tie], (g >= T).astype(np.uint8)[~tie])
    # the phase values are the means of the counts over the phases
    assert c0 == pytest.approx(g[s == 0].mean(), rel=1e-12) or k == 64
    assert abs(c1 - g[s == 1].mean()) <= 1e-9 * c1 or k == 64


@pytest.mark.parametrize("nh", [(3, 2, 2), (2, 3, 2), (2, 2, 3)])
@pytest.mark.parametrize("nu", [0.4, 1.5, 3.0])
def test_reaches_the_brute_force_minimum(nh, nu):
    """On 12-box periodic grids (4096 volumes) the thresholded relaxed
    solution attains the smallest value of the functional for the phase
    values of the first outer iteration (the relaxation is exact for the face
    total variation).  Grids elongated along each axis catch a transposed
    neighbour."""
    nh = np.array(nh)
    rng = np.random.default_rng(int(nu * 10) + int(nh[0]))
    for trial in range(6):
        g = rng.integers(0, 7, 12).astype(np.int32)
        s0 = (g >= 3).astype(np.uint8)
        if s0.all() or not s0.any():
            continue
        s, u, (c0, c1), k = O.ms_segment(g, nh, s0, nu, 6000, 1)
        best = min(O.ms_energy(g, nh, np.array(bits), c0, c1, nu)
                   for bits in itertools.product((0, 1), repeat=12))
        assert O.ms_energy(g, nh, s, c0, c1, nu) <= best + 1e-9, (trial, g)


def test_translation_invariance():
    rng = np.random.default_rng(9)
    nh = np.array([6, 8, 10])
    n = int(np.prod(nh))
    z = np.arange(n) // 48
    g = np.where((z >= 3) & (z < 7), rng.poisson(4.0, n), rng.poisson(0.3, n)).astype(np.int32)
    s0 = (g >= 2).astype(np.uint8)
    s, u, c, k = O.ms_segment(g, nh, s0, 1.8, 300, 4)
    shift = (1, 3, 4)  # x, y, z
    roll = lambda a: np.roll(a.reshape(nh[2], nh[1], nh[0]), (shift[2], shift[1], shift[0]), (0, 1, 2)).ravel()
    s2, u2, c2, k2 = O.ms_segment(roll(g), nh, roll(s0), 1.8, 300, 4)
    assert np.array_equal(s2, roll(s))
    assert np.allclose(u2, roll(u), atol=1e-12)


def test_length_term_removes_noise_bubbles():
    """A slab of Poisson counts (liquid 2.7, vapor 0.07 per box: the slab
    workload's densities at h = 1.5): the plain midpoint threshold of the
    counts leaves a quarter of the liquid boxes in the vapor phase; with the
    length term the liquid is one slab again."""
    rng = np.random.default_rng(5)
    nh = np.array([12, 12, 24])
    n = int(np.prod(nh))
    z = np.arange(n) // 144
    liquid = (z >= 8) & (z < 16)
    g = np.where(liquid, rng.poisson(2.7, n), rng.poisson(0.07, n)).astype(np.int32)
    s0 = liquid.astype(np.uint8)
    plain, _, _, _ = O.ms_segment(g, nh, s0, 0.0, 50, 10)
    assert (plain[liquid] == 0).mean() > 0.15
    s, _, _, _ = O.ms_segment(g, nh, s0, 4.0, 300, 10)
    assert np.array_equal(s, s0)
