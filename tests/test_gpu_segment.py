"""Regularised two-phase segmentation on the GPU (params.segmentation = 1,
Section 2.1) against the oracle's, through the C ABI.

The FP64 form rounds every step as the oracle does (no fused multiply-add),
so the segmented volume, the interface boxes and the threshold are
bit-exact.  The mixed form iterates in FP32: its volume may differ only in
boxes whose relaxed value the oracle leaves within 1e-3 of the threshold 1/2.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1701_05242_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    import paper_1701_05242_gb300.dcm as dcm
    return dcm


def noisy_counts(nh, seed, liquid=2.7, vapor=0.07, waves=0.0):
    """Poisson box counts of a liquid slab in vapor (the slab densities at
    h = 1.5), optionally with a wavy surface."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = nh
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    lo = nz / 3 + waves * np.sin(2 * np.pi * x / nx)
    hi = 2 * nz / 3 + waves * np.cos(2 * np.pi * y / ny)
    liq = (z >= lo) & (z < hi)
    g = np.where(liq, rng.poisson(liquid, liq.shape), rng.poisson(vapor, liq.shape)).astype(np.int32)
    return np.ascontiguousarray(g.transpose(2, 1, 0)).ravel()   # x fastest


def run(D, count, nh, prec, nu, inner, outer, w=0, min_component=0):
    h = 1.5
    box = tuple(n * h for n in nh)
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    p = D.make_params(box, precision=P, smooth_w=w, segmentation=1, ms_nu=nu, ms_inner=inner, ms_outer=outer,
                      min_component=min_component, rc_max=min(6.0, min(box) / 2))
    ctx = D.Context(p)
    bc = torch.from_numpy(count).cuda()
    s = torch.empty(ctx.nbox, dtype=torch.uint8, device="cuda")
    iface = torch.empty_like(s)
    T = torch.empty(1, dtype=torch.int32, device="cuda")
    D.dcm_detect_interface(ctx, bc, s, iface, T)
    torch.cuda.synchronize()
    assert D.dcm_status(ctx) == D.DCM_OK
    return s.cpu().numpy(), iface.cpu().numpy(), int(T.item())


def oracle(count, nh, nu, inner, outer, w=0, min_component=0):
    nh = np.asarray(nh, dtype=np.int64)
    g, T, s0, _ = O.detect_interface(count, nh, w)
    s, u, c, k = O.ms_segment(count, nh, s0, nu, inner, outer)
    if min_component > 0:
        s, _ = O.remove_small_components(s, nh, min_component)
    return s, O.interface(s, nh), T, u


@pytest.mark.parametrize("nh,seed,waves", [((16, 16, 48), 1, 0.0), ((20, 24, 36), 2, 2.5), ((17, 13, 31), 3, 1.0)])
@pytest.mark.parametrize("nu", [0.0, 1.5, 4.0])
def test_fp64_bit_exact(D, nh, seed, waves, nu):
    count = noisy_counts(nh, seed, waves=waves)
    s, iface, T = run(D, count, nh, "fp64", nu, 150, 4)
    so, io, To, _ = oracle(count, nh, nu, 150, 4)
    assert T == To
    assert np.array_equal(s, so) and np.array_equal(iface, io)


@pytest.mark.parametrize("nh,seed", [((16, 16, 48), 4), ((20, 24, 36), 5)])
@pytest.mark.parametrize("nu", [1.5, 4.0])
def test_mixed_agrees_up_to_threshold_ties(D, nh, seed, nu):
    count = noisy_counts(nh, seed, waves=1.5)
    s, iface, T = run(D, count, nh, "mixed", nu, 150, 4)
    so, io, To, u = oracle(count, nh, nu, 150, 4)
    diff = s != so
    near = np.abs(u - 0.5) < 1e-3
    assert np.all(near[diff]), (diff.sum(), near.sum())
    assert diff.sum() <= max(2, 1e-3 * s.size)


def test_length_term_removes_bubbles_and_feeds_the_filter(D):
    """Noisy counts without smoothing (w = 0): the threshold leaves many
    vapor boxes inside the liquid, the length term removes them; with the
    bubble filter after it, the result is the oracle's in FP64."""
    nh = (24, 24, 48)
    count = noisy_counts(nh, 9, waves=2.0)
    s_plain, _, _ = run(D, count, nh, "fp64", 0.0, 50, 4)
    s, iface, _ = run(D, count, nh, "fp64", 4.0, 200, 4)
    nz = nh[2]
    z = np.arange(s.size) // (nh[0] * nh[1])
    core = (z >= nz / 3 + 4) & (z < 2 * nz / 3 - 4)
    assert (s_plain[core] == 0).sum() > 50
    assert (s[core] == 0).sum() == 0
    s2, i2, _ = run(D, count, nh, "fp64", 4.0, 200, 4, min_component=20)
    so, io, _, _ = oracle(count, nh, 4.0, 200, 4, min_component=20)
    assert np.array_equal(s2, so) and np.array_equal(i2, io)


def test_step_with_the_regularised_segmentation(D):
    """The whole timestep with params.segmentation = 1 (interface from the
    regularised segmentation, then distances and cutoffs): it runs, reports
    no device error, and its cutoffs equal the oracle's for the same volume."""
    slab = synth.make_slab(synth.named("slab_1935"))
    p = D.make_params(slab.box, n_max=slab.n, precision=D.DCM_PREC_FP64, recompute_every=1, segmentation=1,
                      ms_nu=4.0, ms_inner=100, ms_outer=3)
    ctx = D.Context(p)
    st = D.State(ctx, D.to_real4(torch.from_numpy(slab.pos), None, torch.float64),
                 D.to_real4(torch.from_numpy(slab.vel), None, torch.float64))
    D.dcm_step_init(ctx, st)
    D.dcm_step(ctx, st, 0.005, 2)
    assert D.dcm_status(ctx) == D.DCM_OK
    pos, _, rc, _ = st.current()
    pos = pos.cpu().numpy()[:, :3]
    nh = O.grid_dims(slab.box, 1.5)
    _, count, _, _ = O.bin_particles(pos, slab.box, 1.5)
    s, iface, _, _ = oracle(count, nh, 4.0, 100, 3, w=2)
    Dd, _ = O.cfsm(s, iface, nh, 1.5, 6.0)
    _, orc = O.cutoffs(pos, Dd, nh, 1.5, 6.0, 3.0, 6.0, 3.0)
    assert np.abs(rc.cpu().numpy() - orc).max() <= 1e-12


def test_segmentation_validation(D):
    for kw in (dict(segmentation=2), dict(segmentation=1, ms_nu=-1.0), dict(segmentation=1, ms_inner=0),
               dict(segmentation=1, ms_outer=65)):
        rc, msg = D.dcm_validate_params(D.make_params((12.0, 12.0, 48.0), **kw))
        assert rc == D.DCM_ERR_INVALID_ARG and msg
    p = D.make_params((1, 1, 1), segmentation=1)
    with pytest.raises(D.DcmError):
        D.Batch(p, [(12.0, 12.0, 48.0)], [10])
