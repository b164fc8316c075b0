"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated once, used below):
  cells, counts, starts, permutation, box sums, threshold, S, interface: bit-exact
  distances D: |dD| <= 1e-5 max(|D|, h) on finite values, identical +inf sets
  cutoffs rc: |drc| <= 2e-6 (the ramp maps dD one to one into drc; FP32 ulp at 6 is 4.8e-7)
  forces (mixed form): sqrt(sum|dF|^2 / sum|F|^2) <= 1e-5
  energy E and virial W (mixed form): relative <= 1e-7
  FP64 form: everything within 1e-12 relative (FP64 against FP64, different summation order)
Pair-inclusion flips (r^2 within rounding of rc^2) are counted; they are bounded
by the pairs lying within 1e-5 relative of a cutoff.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1701_05242_gb300 import synth

pytestmark = pytest.mark.gpu

F_RMS_TOL = 1e-5
EW_TOL = 1e-7
D_TOL = 1e-5
RC_TOL = 2e-6
FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def D():
    import paper_1701_05242_gb300.dcm as dcm
    assert torch.cuda.is_available()
    return dcm


def make_ctx(D, box, n_max, precision=None, **kw):
    prec = D.DCM_PREC_MIXED if precision is None else precision
    p = D.make_params(box, n_max=int(n_max), precision=prec, **kw)
    return D.Context(p)


def real_of(D, prec):
    return torch.float32 if prec == D.DCM_PREC_MIXED else torch.float64


def pos4_of(D, pos, types, prec):
    return D.to_real4(torch.from_numpy(np.asarray(pos, np.float32)),
                      None if types is None else torch.from_numpy(np.asarray(types)), real_of(D, prec))


def gpu_bin(D, ctx, pos4):
    n = pos4.shape[0]
    dev = pos4.device
    cell = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    start = torch.empty(ctx.ncell + 1, dtype=torch.int32, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ps = torch.empty_like(pos4) if n else torch.empty((1, 4), dtype=pos4.dtype, device=dev)
    D.dcm_bin(ctx, n, pos4 if n else ps, cell, start, perm, ps)
    torch.cuda.synchronize()
    return cell[:n].cpu().numpy(), start.cpu().numpy(), perm[:n].cpu().numpy(), ps[:n]


def assert_distances(Dg, Do, r_grid, tol):
    """Finite values within tol * max(D, h); the +inf sets agree except at the
    acceptance threshold r_grid, where FP32 and FP64 may round a value of about
    r_grid to either side."""
    fin = np.isfinite(Do) & np.isfinite(Dg)
    flip = np.isfinite(Do) != np.isfinite(Dg)
    other = np.where(np.isfinite(Do), Do, Dg)
    assert np.all(other[flip] >= r_grid * (1 - tol)), other[flip].min() if flip.any() else None
    assert flip.sum() <= max(2, 1e-4 * flip.size)
    assert np.all(np.abs(Dg[fin] - Do[fin]) <= tol * np.maximum(Do[fin], 1.5))


def rms_rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def near_cutoff_pairs(pos, rc, box, idx=None, rel=1e-5):
    """Ordered pairs (i, j) with |r_ij^2 - rc_i^2| <= rel rc_i^2 (possible inclusion flips)."""
    pos = np.asarray(pos, np.float64)
    box = np.asarray(box, np.float64)
    if idx is None and len(pos) > 5000:
        from scipy.spatial import cKDTree
        t = cKDTree(np.mod(pos, box), boxsize=box)
        q = np.mod(pos, box)
        outer = t.query_ball_point(q, np.sqrt(1 + rel) * rc, return_length=True)
        inner = t.query_ball_point(q, np.sqrt(1 - rel) * rc, return_length=True)
        return int((outer - inner).sum())
    count = 0
    for i in (range(len(pos)) if idx is None else idx):
        d = pos[i] - pos
        d -= box * np.round(d / box)
        r2 = (d * d).sum(1)
        r2[i] = -1
        count += int((np.abs(r2 - rc[i] ** 2) <= rel * rc[i] ** 2).sum())
    return count


# --------------------------------------------------------------------------- binning
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("l", [1.5, 0.75])
def test_bin_bit_exact(D, slab_1935, prec, l):
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    ctx = make_ctx(D, slab_1935.box, slab_1935.n, P, l=l)
    pos4 = pos4_of(D, slab_1935.pos, None, P)
    cell, start, perm, ps = gpu_bin(D, ctx, pos4)
    oc, ocount, ostart, operm = O.bin_particles(slab_1935.pos, slab_1935.box, l)
    assert np.array_equal(cell, oc)
    assert np.array_equal(start, ostart)
    assert np.array_equal(perm, operm)
    assert torch.equal(ps.cpu(), pos4.cpu()[torch.from_numpy(operm).long()])


def test_bin_edges_and_empty(D):
    box = (12.0, 12.0, 12.0)
    l = 1.5
    xs = [0.0, 1.5, np.nextafter(np.float32(1.5), np.float32(0)), 3.0, 10.5, np.nextafter(np.float32(12), np.float32(0)),
          6.0, 7.5]
    pts = np.array([[x, y, z] for x in xs for y in xs[:3] for z in xs[-3:]], np.float32)
    ctx = make_ctx(D, box, len(pts) + 10)
    pos4 = pos4_of(D, pts, None, D.DCM_PREC_MIXED)
    cell, start, perm, _ = gpu_bin(D, ctx, pos4)
    oc, _, ostart, operm = O.bin_particles(pts, box, l)
    assert np.array_equal(cell, oc) and np.array_equal(start, ostart) and np.array_equal(perm, operm)
    # all particles in one cell keep their input order
    same = np.full((37, 3), 4.0, np.float32) + np.linspace(0, 1.0, 37, dtype=np.float32)[:, None] * 0.4
    cell, start, perm, _ = gpu_bin(D, ctx, pos4_of(D, same, None, D.DCM_PREC_MIXED))
    assert np.array_equal(perm, np.arange(37)) and len(set(cell.tolist())) == 1
    # no particles
    cell, start, perm, _ = gpu_bin(D, ctx, torch.empty((0, 4), device="cuda"))
    assert start.max() == 0 and start.shape[0] == ctx.ncell + 1


@pytest.mark.parametrize("box,lx", [((60.0, 45.0, 30.0), 0.0), ((60.0, 45.0, 30.0), 0.5), ((61.5, 45.0, 31.5), 0.0)])
def test_bin_many_scan_tiles(D, box, lx):
    """Binning whose cell-count scan spans several look-back tiles of 8,192
    cells with a ragged last tile (24,000, 72,000 and 25,830 cells, the last
    not a multiple of a thread's 16 cells nor of 4), with uniform particles,
    a dense clump in one cell and empty regions: cells, starts and order
    bit-exact against the oracle."""
    rng = np.random.default_rng(11)
    uni = rng.random((40000, 3)) * np.array(box)
    clump = np.array([30.2, 20.1, 10.3]) + rng.random((700, 3)) * 0.2
    half = rng.random((9000, 3)) * np.array([30.0, 45.0, 15.0])
    uni = np.minimum(uni, np.nextafter(np.array(box, np.float32), np.float32(0)))
    pts = np.concatenate([uni, clump, half]).astype(np.float32)
    ctx = make_ctx(D, box, len(pts), lx=lx)
    edges = (lx if lx > 0 else 1.5, 1.5, 1.5)
    assert ctx.ncell == int(np.prod(O.grid_dims(box, edges))) and ctx.ncell % 8192 != 0 and ctx.ncell > 2 * 8192
    cell, start, perm, ps = gpu_bin(D, ctx, pos4_of(D, pts, None, D.DCM_PREC_MIXED))
    oc, _, ostart, operm = O.bin_particles(pts, box, edges)
    assert np.array_equal(cell, oc) and np.array_equal(start, ostart) and np.array_equal(perm, operm)
    assert D.dcm_status(ctx) == D.DCM_OK


def test_scan_wait_runs_out_and_the_context_stays_usable(D, slab_1935):
    """The scan's look-back wait for a tile that never publishes runs out
    with DCM_ERR_TIMEOUT (no fault, no hang); the same context then bins
    bit-exactly."""
    ctx = make_ctx(D, slab_1935.box, slab_1935.n)
    assert D.dcm_scan_wait_selftest(ctx) == D.DCM_ERR_TIMEOUT
    assert D.dcm_status(ctx) == D.DCM_OK
    cell, start, perm, _ = gpu_bin(D, ctx, pos4_of(D, slab_1935.pos, None, D.DCM_PREC_MIXED))
    oc, _, ostart, operm = O.bin_particles(slab_1935.pos, slab_1935.box, 1.5)
    assert np.array_equal(cell, oc) and np.array_equal(start, ostart) and np.array_equal(perm, operm)


def test_capacity_error(D, slab_1935):
    ctx = make_ctx(D, slab_1935.box, 100)
    pos4 = pos4_of(D, slab_1935.pos, None, D.DCM_PREC_MIXED)
    with pytest.raises(D.DcmError) as e:
        gpu_bin(D, ctx, pos4)
    assert e.value.code == D.DCM_ERR_CAPACITY


# ------------------------------------------------------------------- detection
def gpu_detect(D, ctx, pos4):
    n = pos4.shape[0]
    bc = torch.empty(ctx.nbox, dtype=torch.int32, device="cuda")
    D.dcm_box_counts(ctx, n, pos4, bc)
    s = torch.empty(ctx.nbox, dtype=torch.uint8, device="cuda")
    iface = torch.empty_like(s)
    T = torch.empty(1, dtype=torch.int32, device="cuda")
    g = torch.empty(ctx.nbox, dtype=torch.int32, device="cuda")
    D.dcm_detect_interface(ctx, bc, s, iface, T, g)
    torch.cuda.synchronize()
    return bc.cpu().numpy(), g.cpu().numpy(), int(T.item()), s, iface


@pytest.mark.parametrize("w,thr", [(2, -1), (1, -1), (0, -1), (2, 160)])
def test_detect_bit_exact(D, slab_1935, w, thr):
    ctx = make_ctx(D, slab_1935.box, slab_1935.n, smooth_w=w, threshold=thr)
    pos4 = pos4_of(D, slab_1935.pos, None, D.DCM_PREC_MIXED)
    bc, g, T, s, iface = gpu_detect(D, ctx, pos4)
    nh = O.grid_dims(slab_1935.box, 1.5)
    _, ocount, _, _ = O.bin_particles(slab_1935.pos, slab_1935.box, 1.5)
    og, oT, os_, oif = O.detect_interface(ocount, nh, w, None if thr < 0 else thr)
    assert np.array_equal(bc, ocount)
    assert np.array_equal(g, og)
    assert T == oT
    assert np.array_equal(s.cpu().numpy(), os_) and np.array_equal(iface.cpu().numpy(), oif)


def test_detect_single_phase_has_no_interface(D):
    box = (13.5, 13.5, 13.5)                   # 9 boxes per dimension
    rng = np.random.default_rng(0)
    pts = rng.uniform(0, 13.5, size=(2000, 3)).astype(np.float32)
    ctx = make_ctx(D, box, 2000, smooth_w=4)   # 9-wide box sum covers the periodic grid once: all equal
    _, g, T, s, iface = gpu_detect(D, ctx, pos4_of(D, pts, None, D.DCM_PREC_MIXED))
    assert len(set(g.tolist())) == 1 and g[0] == 2000
    assert T == g[0] + 1 and int(iface.sum()) == 0 and int(s.sum()) == 0


# -------------------------------------------------------------------- distance
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_distance(D, slab_1935, prec):
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    ctx = make_ctx(D, slab_1935.box, slab_1935.n, P)
    pos4 = pos4_of(D, slab_1935.pos, None, P)
    _, _, _, s, iface = gpu_detect(D, ctx, pos4)
    Dg = torch.empty(ctx.nbox, dtype=real_of(D, P), device="cuda")
    it = torch.empty(1, dtype=torch.int32, device="cuda")
    D.dcm_distance(ctx, s, iface, Dg, it)
    Dg = Dg.cpu().numpy().astype(np.float64)
    nh = O.grid_dims(slab_1935.box, 1.5)
    Dj, itj = O.distance_jacobi(s.cpu().numpy(), iface.cpu().numpy(), nh, 1.5, 6.0)
    tol = D_TOL if P == D.DCM_PREC_MIXED else FP64_TOL
    assert_distances(Dg, Dj, 6.0, tol)
    assert abs(int(it.item()) - itj) <= (2 if P == D.DCM_PREC_MIXED else 0)


@pytest.mark.parametrize("seed", [0, 1])
def test_distance_random_blobs(D, seed):
    # hand-built S / interface volumes exercising diagonal fronts
    rng = np.random.default_rng(seed)
    box = (21.0, 18.0, 24.0)
    nh = O.grid_dims(box, 1.5)
    nb = int(np.prod(nh))
    s = np.ones(nb, np.uint8)
    iface = (rng.random(nb) < 0.004).astype(np.uint8)
    s[rng.random(nb) < 0.002] = 0
    ctx = make_ctx(D, box, 16, rc_min=3.0, rc_max=6.0, r_grid=7.5)
    Dg = torch.empty(nb, dtype=torch.float32, device="cuda")
    it = torch.empty(1, dtype=torch.int32, device="cuda")
    D.dcm_distance(ctx, torch.from_numpy(s).cuda(), torch.from_numpy(iface).cuda(), Dg, it)
    Dj, itj = O.distance_jacobi(s, iface, nh, 1.5, 7.5)
    Dg = Dg.cpu().numpy().astype(np.float64)
    assert_distances(Dg, Dj, 7.5, D_TOL)
    # FP32 and FP64 sweeps may settle their last ulps one sweep apart
    assert abs(int(it.item()) - itj) <= 2


def test_distance_not_converged_reports(D):
    box = (6.0, 6.0, 60.0)
    nh = O.grid_dims(box, 1.5)
    nb = int(np.prod(nh))
    s = np.ones(nb, np.uint8)
    iface = np.zeros(nb, np.uint8)
    iface[:16] = 1
    ctx = make_ctx(D, box, 16, rc_min=1.5, rc_max=3.0, r_grid=100.0, iter_max=3)
    Dg = torch.empty(nb, dtype=torch.float32, device="cuda")
    with pytest.raises(D.DcmError) as e:
        D.dcm_distance(ctx, torch.from_numpy(s).cuda(), torch.from_numpy(iface).cuda(), Dg)
    assert e.value.code == D.DCM_ERR_NOT_CONVERGED
    assert D.dcm_status(ctx) == D.DCM_ERR_NOT_CONVERGED
    assert D.dcm_status(ctx) == D.DCM_OK   # cleared by the read


# --------------------------------------------------------------------- cutoffs
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_cutoffs(D, slab_1935, prec):
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    ctx = make_ctx(D, slab_1935.box, slab_1935.n, P)
    pos4 = pos4_of(D, slab_1935.pos, None, P)
    _, _, _, s, iface = gpu_detect(D, ctx, pos4)
    Dg = torch.empty(ctx.nbox, dtype=real_of(D, P), device="cuda")
    D.dcm_distance(ctx, s, iface, Dg)
    rc = torch.empty(slab_1935.n, dtype=real_of(D, P), device="cuda")
    D.dcm_cutoffs(ctx, slab_1935.n, pos4, Dg, rc)
    p = O.Params(box=slab_1935.box)
    a = O.assign_cutoffs(slab_1935.pos, p)
    tol = RC_TOL if P == D.DCM_PREC_MIXED else FP64_TOL * 6
    assert np.abs(rc.cpu().numpy().astype(np.float64) - a["rc"]).max() <= tol


# ---------------------------------------------------------------------- forces
def forces_case(D, slab, prec, rc64, types=None, eps=(1.0,), sigma=(1.0,), shift=0, l=1.5, box=None, kernel=0,
                acc=0):
    box = slab.box if box is None else box
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    kw = dict(ntypes=len(eps), eps=eps, sigma=sigma, shift_energy=shift, l=l, force_kernel=kernel, accumulation=acc)
    ctx = make_ctx(D, box, slab.n, P, **kw)
    real = real_of(D, P)
    rc_in = rc64.astype(np.float32).astype(np.float64) if P == D.DCM_PREC_MIXED else rc64
    pos4 = pos4_of(D, slab.pos, types, P)
    cell, start, perm, ps = gpu_bin(D, ctx, pos4)
    rcs = torch.from_numpy(rc_in[perm]).to(real).cuda()
    F = torch.empty_like(ps)
    tot = torch.zeros(3, dtype=torch.float64, device="cuda")
    D.dcm_forces(ctx, slab.n, ps, rcs, torch.from_numpy(start).cuda(), F, tot)
    torch.cuda.synchronize()
    Fs = F.cpu().numpy().astype(np.float64)
    Fg = np.empty_like(Fs)
    Fg[perm] = Fs
    ref = O.forces_cells(slab.pos, rc_in, box, l, types, eps, sigma, bool(shift))
    return Fg, tot.cpu().numpy(), ref, rc_in


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("l", [1.5, 1.0])
def test_forces_dcm_cutoffs(D, slab_1935, prec, l):
    p = O.Params(box=slab_1935.box)
    rc64 = O.assign_cutoffs(slab_1935.pos, p)["rc"]
    Fg, tot, ref, rc_in = forces_case(D, slab_1935, prec, rc64, l=l)
    if prec == "mixed":
        assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
        assert abs(tot[0] - ref.E) <= EW_TOL * abs(ref.E)
        assert abs(tot[1] - ref.W) <= EW_TOL * abs(ref.W)
        assert abs(Fg[:, 3] - ref.e).max() <= 1e-5 * np.abs(ref.e).max()
        assert abs(int(tot[2]) - ref.npairs) <= near_cutoff_pairs(slab_1935.pos, rc_in, slab_1935.box)
    else:
        assert np.abs(Fg[:, :3] - ref.F).max() <= FP64_TOL * np.abs(ref.F).max()
        assert abs(tot[0] - ref.E) <= FP64_TOL * abs(ref.E)
        assert abs(tot[1] - ref.W) <= FP64_TOL * abs(ref.W)
        assert int(tot[2]) == ref.npairs


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_forces_uniform_and_shift(D, slab_1935, prec):
    rc64 = np.full(slab_1935.n, 4.5)
    Fg, tot, ref, _ = forces_case(D, slab_1935, prec, rc64, shift=1)
    tol = F_RMS_TOL if prec == "mixed" else FP64_TOL
    assert rms_rel(Fg[:, :3], ref.F) <= tol
    assert abs(tot[0] - ref.E) <= (EW_TOL if prec == "mixed" else FP64_TOL) * abs(ref.E)
    # uniform cutoff: Newton's third law makes the net force vanish (to rounding)
    assert np.abs(Fg[:, :3].sum(0)).max() <= (1e-5 if prec == "mixed" else 1e-10) * np.abs(Fg[:, :3]).sum()


@pytest.mark.parametrize("prec,kernel,shift,acc", [("mixed", 1, 0, 0), ("mixed", 3, 0, 0), ("mixed", 3, 1, 0),
                                                   ("mixed", 3, 0, 1), ("mixed", 3, 1, 2), ("mixed", 3, 0, 3),
                                                   ("mixed", 3, 0, 4), ("mixed", 3, 1, 5), ("mixed", 3, 1, 6),
                                                   ("mixed", 1, 1, 2), ("mixed", 1, 0, 7), ("fp64", 0, 0, 0)])
def test_forces_two_types(D, prec, kernel, shift, acc):
    """Two types with Lorentz-Berthelot mixing: the scalar loop (kernel 1),
    the packed typed loop (kernel 3, also with the shifted energy), each
    per-particle accumulation form, and FP64."""
    spec = synth.named("slab_256k_2types")
    spec.box = (18.0, 18.0, 72.0)
    slab = synth.make_slab(spec)
    rng = np.random.default_rng(3)
    rc64 = rng.uniform(3.0, 6.0, slab.n)
    Fg, tot, ref, rc_in = forces_case(D, slab, prec, rc64, types=slab.types, eps=(1.0, 0.8), sigma=(1.0, 1.1),
                                      kernel=kernel, shift=shift, acc=acc)
    if prec == "mixed":
        assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
        assert abs(tot[0] - ref.E) <= EW_TOL * abs(ref.E)
        assert abs(tot[1] - ref.W) <= EW_TOL * abs(ref.W)
        assert np.abs(Fg[:, 3] - ref.e).max() <= 1e-5 * np.abs(ref.e).max()
        assert abs(int(tot[2]) - ref.npairs) <= near_cutoff_pairs(slab.pos, rc_in, slab.box)
    else:
        assert np.abs(Fg[:, :3] - ref.F).max() <= FP64_TOL * np.abs(ref.F).max()
        assert int(tot[2]) == ref.npairs


@pytest.mark.parametrize("shift", [0, 1])
@pytest.mark.parametrize("kernel", [1, 3])
def test_forces_one_type_scaled(D, slab_1935, kernel, shift):
    """One type with eps and sigma other than 1: the scalar loop and the
    packed typed loop (both columns of its row equal).  With sigma = 1.05 the
    0.85 placement puts pairs at 0.81 sigma, deep in the repulsive wall, and
    a few pair energies of ~30 dominate E; each carries the FP32 rounding of
    (sigma^2 / r^2)^6 (a dozen roundings of 2^-24), which does not average
    out over so few terms, so E and W are held to 32 u32 sum |e_i| (and the
    same relative share for W) instead of the 1e-7 of the sigma = 1 slabs."""
    p = O.Params(box=slab_1935.box)
    rc64 = O.assign_cutoffs(slab_1935.pos, p)["rc"]
    Fg, tot, ref, rc_in = forces_case(D, slab_1935, "mixed", rc64, eps=(0.9,), sigma=(1.05,), shift=shift,
                                      kernel=kernel)
    u32 = 2.0 ** -24
    bound = 32 * u32 * np.abs(ref.e).sum()
    print(f"ERR scaled one type kernel {kernel} shift {shift}: E {abs(tot[0] - ref.E) / abs(ref.E):.3g} "
          f"W {abs(tot[1] - ref.W) / abs(ref.W):.3g} (rel), bound {bound / abs(ref.E):.3g}")
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
    assert abs(tot[0] - ref.E) <= bound
    assert abs(tot[1] - ref.W) <= bound / abs(ref.E) * abs(ref.W)
    assert np.abs(Fg[:, 3] - ref.e).max() <= 1e-5 * np.abs(ref.e).max()


@pytest.mark.parametrize("acc", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("kernel", [1, 3])
@pytest.mark.parametrize("l", [1.5, 1.0])
def test_forces_kernel_variants(D, slab_1935, kernel, l, acc):
    """Both cell-list force kernels, in every per-particle accumulation form,
    against the oracle (mixed, one type)."""
    p = O.Params(box=slab_1935.box)
    rc64 = O.assign_cutoffs(slab_1935.pos, p)["rc"]
    Fg, tot, ref, rc_in = forces_case(D, slab_1935, "mixed", rc64, l=l, kernel=kernel, acc=acc)
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
    assert abs(tot[0] - ref.E) <= EW_TOL * abs(ref.E)
    assert abs(tot[1] - ref.W) <= EW_TOL * abs(ref.W)
    assert abs(Fg[:, 3] - ref.e).max() <= 1e-5 * np.abs(ref.e).max()
    assert abs(int(tot[2]) - ref.npairs) <= near_cutoff_pairs(slab_1935.pos, rc_in, slab_1935.box)
    # uniform cutoff with the shifted energy
    Fg, tot, ref, _ = forces_case(D, slab_1935, "mixed", np.full(slab_1935.n, 4.5), shift=1, l=l, kernel=kernel,
                                  acc=acc)
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
    assert abs(tot[0] - ref.E) <= EW_TOL * abs(ref.E)


@pytest.mark.parametrize("lx", [0.75, 0.5])
def test_binning_with_a_finer_row_edge(D, slab_1935, lx):
    """Cells of lx x 1.5 x 1.5 (finer along the contiguous rows): binning
    bit-exact against the oracle's per-axis floor and stable order."""
    ctx = make_ctx(D, slab_1935.box, slab_1935.n, lx=lx)
    assert ctx.ncell == int(np.prod(O.grid_dims(slab_1935.box, (lx, 1.5, 1.5))))
    cell, start, perm, ps = gpu_bin(D, ctx, pos4_of(D, slab_1935.pos, None, D.DCM_PREC_MIXED))
    oc, ocount, ostart, operm = O.bin_particles(slab_1935.pos, slab_1935.box, (lx, 1.5, 1.5))
    assert np.array_equal(cell, oc) and np.array_equal(start, ostart) and np.array_equal(perm, operm)


@pytest.mark.parametrize("kernel", [1, 3])
@pytest.mark.parametrize("lx", [0.75, 0.5])
def test_forces_with_a_finer_row_edge(D, slab_1935, kernel, lx):
    """Every cell-list kernel on cells of lx x 1.5 x 1.5 against the oracle
    (whose result does not depend on the cells)."""
    p = O.Params(box=slab_1935.box)
    rc64 = O.assign_cutoffs(slab_1935.pos, p)["rc"]
    box = slab_1935.box
    ctx = make_ctx(D, box, slab_1935.n, lx=lx, force_kernel=kernel)
    rc_in = rc64.astype(np.float32).astype(np.float64)
    cell, start, perm, ps = gpu_bin(D, ctx, pos4_of(D, slab_1935.pos, None, D.DCM_PREC_MIXED))
    F = torch.empty_like(ps)
    tot = torch.zeros(3, dtype=torch.float64, device="cuda")
    D.dcm_forces(ctx, slab_1935.n, ps, torch.from_numpy(rc_in[perm]).float().cuda(), torch.from_numpy(start).cuda(),
                 F, tot)
    torch.cuda.synchronize()
    Fg = np.empty((slab_1935.n, 4))
    Fg[perm] = F.cpu().numpy()
    tot = tot.cpu().numpy()
    ref = O.forces_cells(slab_1935.pos, rc_in, box, 1.5)
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
    assert abs(tot[0] - ref.E) <= EW_TOL * abs(ref.E)
    assert abs(tot[1] - ref.W) <= EW_TOL * abs(ref.W)
    assert abs(int(tot[2]) - ref.npairs) <= near_cutoff_pairs(slab_1935.pos, rc_in, box)


FAR = np.array([[1.0e4, 5.0, 5.0], [-1.0e4, 6.0, 20.0], [3.0, 5.0e3, 30.0], [7.0, -3.0e3, 10.0],
                [2.0, 2.0, 1.0e5], [4.0, 9.0, -2.0e4], [1.0e30, 1.0, 1.0], [-1.0e30, -1.0e30, 40.0]], np.float32)


@pytest.mark.parametrize("kernel,lx", [(1, 0.0), (3, 0.0), (3, 0.75), (1, 0.5), (3, 0.5)])
def test_coordinates_outside_the_box(D, slab_1935, kernel, lx):
    """Finite coordinates far outside [0, L) are binned into the boundary
    cells: every kernel keeps its indices in range, the far particles accept
    no pair, and the others get the forces of the system without them."""
    n0 = slab_1935.n
    pos = np.concatenate([slab_1935.pos.astype(np.float32), FAR])
    n = len(pos)
    rc64 = O.assign_cutoffs(slab_1935.pos, O.Params(box=slab_1935.box))["rc"]
    rc = np.concatenate([rc64, np.full(len(FAR), 6.0)]).astype(np.float32)
    ctx = make_ctx(D, slab_1935.box, n, force_kernel=kernel, lx=lx)
    cell, start, perm, ps = gpu_bin(D, ctx, pos4_of(D, pos, None, D.DCM_PREC_MIXED))
    F = torch.empty_like(ps)
    tot = torch.zeros(3, dtype=torch.float64, device="cuda")
    rcs = torch.from_numpy(rc[perm]).cuda()
    starts = torch.from_numpy(start).cuda()
    D.dcm_forces(ctx, n, ps, rcs, starts, F, tot)
    torch.cuda.synchronize()
    Fg = np.empty((n, 4))
    Fg[perm] = F.cpu().numpy()
    rc_in = rc[:n0].astype(np.float64)
    ref = O.forces_cells(slab_1935.pos, rc_in, slab_1935.box, 1.5)
    assert np.all(Fg[n0:] == 0.0)
    assert rms_rel(Fg[:n0, :3], ref.F) <= F_RMS_TOL
    assert abs(int(tot[2].item()) - ref.npairs) <= near_cutoff_pairs(slab_1935.pos, rc_in, slab_1935.box)
    if kernel == 1:  # the adjoint walks the same rows
        A = torch.zeros_like(ps)
        A[:, :3] = 2 * F[:, :3]
        G = torch.empty_like(ps)
        dpar = torch.zeros(4, dtype=torch.float64, device="cuda")
        D.dcm_forces_backward(ctx, n, ps, rcs, starts, A, 1.0, G, dpar)
        torch.cuda.synchronize()
        assert np.isfinite(G.cpu().numpy()).all() and np.isfinite(dpar.cpu().numpy()).all()
    assert D.dcm_status(ctx) == D.DCM_OK


@pytest.mark.parametrize("skin", [0.0, 0.4])
def test_step_with_coordinates_outside_the_box(D, slab_1935, skin):
    """Steps (cell path, and Verlet lists whose build walks the same rows)
    with particles far outside the box: no error, finite thermodynamics, and
    the far particles feel no force."""
    pos = np.concatenate([slab_1935.pos.astype(np.float32), FAR])
    vel = np.concatenate([slab_1935.vel.astype(np.float32), np.zeros_like(FAR)])
    n = len(pos)
    ctx = make_ctx(D, slab_1935.box, n, recompute_every=5, skin=skin, rc_max=5.5)
    st = D.State(ctx, pos4_of(D, pos, None, D.DCM_PREC_MIXED),
                 D.to_real4(torch.from_numpy(vel), None, torch.float32))
    D.dcm_step_init(ctx, st)
    for _ in range(12):
        D.dcm_step(ctx, st, 0.005, 1)
    th = st.thermo.cpu().numpy()
    assert D.dcm_status(ctx) == D.DCM_OK
    assert np.isfinite(th).all()
    p, v, _, ids = st.current()
    far = ids.cpu().numpy() >= slab_1935.n
    assert far.sum() == len(FAR)
    assert np.all(v.cpu().numpy()[far, :3] == 0.0)


@pytest.mark.parametrize("k", [-1, 2, 4, 5, 6])
def test_forces_kernel_rejects_unknown(D, k):
    with pytest.raises(D.DcmError):
        make_ctx(D, (12.0, 12.0, 48.0), 10, force_kernel=k)


@pytest.mark.parametrize("a", [-1, 8])
def test_accumulation_rejects_unknown(D, a):
    with pytest.raises(D.DcmError):
        make_ctx(D, (12.0, 12.0, 48.0), 10, accumulation=a)


def test_accumulation_resolution(D):
    """AUTO runs the plane Kahan form; the FP64 form ignores the field;
    the scalar kernel runs the row form of a pair form."""
    box = (12.0, 12.0, 48.0)
    assert D.dcm_accumulation(make_ctx(D, box, 10)) == D.DCM_ACC_PLANE_KAHAN
    assert D.dcm_accumulation(make_ctx(D, box, 10, accumulation=D.DCM_ACC_PAIR_FP64)) == D.DCM_ACC_PAIR_FP64
    assert D.dcm_accumulation(make_ctx(D, box, 10, D.DCM_PREC_FP64, accumulation=4)) == D.DCM_ACC_FP32
    assert D.dcm_accumulation(make_ctx(D, box, 10, force_kernel=1, accumulation=4)) == D.DCM_ACC_ROW_KAHAN
    assert D.dcm_accumulation(make_ctx(D, box, 10, force_kernel=1, accumulation=5)) == D.DCM_ACC_ROW_FP64


@pytest.mark.parametrize("kernel", [1, 3])
def test_forces_tiny_box_and_ragged_kernels(D, kernel):
    """rc_max = L/2 (rows reaching both periodic images), 97 particles,
    some cutoffs 0 (no pairs, no shift)."""
    rng = np.random.default_rng(12)
    box = (12.0, 12.0, 12.0)
    pts = rng.uniform(0, 12, size=(97, 3)).astype(np.float32)

    class S:
        pass
    s = S()
    s.pos, s.n, s.box = pts, 97, box
    rc64 = rng.choice([0.0, 3.0, 4.5, 6.0], 97)
    Fg, tot, ref, rc_in = forces_case(D, s, "mixed", rc64, kernel=kernel, shift=1)
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
    # uniform random points: a few overlapping pairs dominate E.  FP32 sums of
    # at most ~50 terms per particle and 32 particles per warp partial:
    # |dE| <= 64 u32 sum|e_i|, u32 = 2^-24
    assert abs(tot[0] - ref.E) <= 64 * 2.0 ** -24 * np.abs(ref.e).sum()
    assert int(tot[2]) == ref.npairs
    assert np.isfinite(Fg).all()


def test_forces_tiny_box_and_ragged(D):
    # rc_max = L/2 exactly (images on both sides), few particles, empty cells
    rng = np.random.default_rng(11)
    box = (12.0, 12.0, 12.0)
    pts = rng.uniform(0, 12, size=(97, 3)).astype(np.float32)

    class S:
        pass
    s = S()
    s.pos, s.n, s.box = pts, 97, box
    rc64 = rng.choice([3.0, 4.5, 6.0], 97)
    Fg, tot, ref, rc_in = forces_case(D, s, "fp64", rc64)
    assert np.abs(Fg[:, :3] - ref.F).max() <= FP64_TOL * np.abs(ref.F).max()
    assert int(tot[2]) == ref.npairs
    Fg, tot, ref, rc_in = forces_case(D, s, "mixed", rc64)
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL


# ------------------------------------------------------------------------ step
def run_gpu_steps(D, slab, P, nsteps, dt=0.005, K=1, per_step=True, lx=0.0):
    ctx = make_ctx(D, slab.box, slab.n, P, recompute_every=K, lx=lx)
    real = real_of(D, P)
    pos4 = pos4_of(D, slab.pos, None, P)
    vel4 = D.to_real4(torch.from_numpy(slab.vel), None, real)
    st = D.State(ctx, pos4, vel4)
    D.dcm_step_init(ctx, st)
    out = [st.thermo.cpu().numpy().copy()]
    for _ in range(nsteps if per_step else 1):
        D.dcm_step(ctx, st, dt, 1 if per_step else nsteps)
        out.append(st.thermo.cpu().numpy().copy())
    assert D.dcm_status(ctx) == D.DCM_OK
    return ctx, st, np.array(out)


@pytest.mark.parametrize("lx", [0.0, 0.75])
def test_step_fp64_matches_oracle_trajectory(D, slab_1935, lx):
    # lx = 0.75: force cells of 0.75 x 1.5 x 1.5 (binning, walk and the
    # separate density histogram), the same trajectory
    nsteps = 30
    ctx, st, th = run_gpu_steps(D, slab_1935, D.DCM_PREC_FP64, nsteps, K=1, lx=lx)
    p = O.Params(box=slab_1935.box, recompute_every=1)
    ost = O.init_state(slab_1935.pos, slab_1935.vel, p)
    assert th[0, 0] == pytest.approx(ost.E, rel=1e-9)
    assert th[0, 2] == pytest.approx(O.kinetic(slab_1935.vel.astype(np.float64)), rel=1e-12)
    for k in range(nsteps):
        ost = O.step(ost, 0.005, p)
        assert th[k + 1, 0] == pytest.approx(ost.E, rel=1e-9), k
        assert th[k + 1, 1] == pytest.approx(ost.W, rel=1e-9), k
        assert th[k + 1, 2] == pytest.approx(O.kinetic(ost.vel), rel=1e-9), k
    pos, vel, rc, ids = st.current()
    ids = ids.cpu().numpy()
    gp = np.empty((slab_1935.n, 3))
    gp[ids] = pos.cpu().numpy()[:, :3]
    d = np.abs(gp - ost.pos)
    d = np.minimum(d, np.array(slab_1935.box) - d)
    assert d.max() <= 1e-9


def test_step_mixed_on_shared_inputs(D, slab_1935):
    # one FP32 step; then the oracle re-evaluates forces at the GPU's own
    # positions and cutoffs (shared inputs), since trajectories diverge
    ctx, st, th = run_gpu_steps(D, slab_1935, D.DCM_PREC_MIXED, 3, K=1)
    pos, vel, rc, ids = st.current()
    pos = pos.cpu().numpy().astype(np.float64)
    rcn = rc.cpu().numpy().astype(np.float64)
    ref = O.forces_cells(pos[:, :3], rcn, slab_1935.box, 1.5)
    Fg = st.force.cpu().numpy().astype(np.float64)
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
    assert abs(th[-1, 0] - ref.E) <= EW_TOL * abs(ref.E)
    # cutoffs recomputed at these positions
    a = O.assign_cutoffs(pos[:, :3], O.Params(box=slab_1935.box))
    assert np.abs(rcn - a["rc"]).max() <= RC_TOL


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_step_batched_call_equals_single_calls(D, slab_1935, prec):
    # one call of 12 steps (the second half kicks fused into the next steps'
    # kick-drift, thermo of the last step only, and in the mixed form force-only
    # evaluations before it) == 12 calls of one step, bit for bit, forces and
    # per-particle energies of the last step included
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    _, st1, th1 = run_gpu_steps(D, slab_1935, P, 12, K=5, per_step=True)
    _, st2, th2 = run_gpu_steps(D, slab_1935, P, 12, K=5, per_step=False)
    assert np.array_equal(th1[-1], th2[-1])
    assert torch.equal(st1.current()[0], st2.current()[0])
    assert torch.equal(st1.current()[1], st2.current()[1])
    assert torch.equal(st1.force, st2.force)
    assert abs(st2.force[:, 3].double().sum().item() - th2[-1][0]) <= 1e-6 * abs(th2[-1][0])


def test_jobs_on_two_states_and_a_copy_stream(D, slab_1935):
    """A stream of jobs as an end-to-end user runs them: two States share one
    context, each job copies its state in from pinned host memory on a copy
    stream, runs dcm_step_init + 10 timesteps on the compute stream and copies
    state and thermo back out; the copies of neighbouring jobs overlap the
    compute.  Every job must give, bit for bit, what one State stepped alone
    gives for the same input."""
    P = D.DCM_PREC_MIXED
    ctx = make_ctx(D, slab_1935.box, slab_1935.n, P, recompute_every=10, lx=0.75)
    pos_h = D.to_real4(torch.from_numpy(slab_1935.pos), None, torch.float32, "cpu").pin_memory()
    vel_h = D.to_real4(torch.from_numpy(slab_1935.vel), None, torch.float32, "cpu").pin_memory()
    ref = D.State(ctx, pos_h.cuda(), vel_h.cuda())
    D.dcm_step_init(ctx, ref)
    D.dcm_step(ctx, ref, 0.005, 10)
    torch.cuda.synchronize()
    rp, rv = ref.current()[0].cpu(), ref.current()[1].cpu()
    rt = ref.thermo.cpu()
    sts = [D.State(ctx, pos_h.cuda(), vel_h.cuda()) for _ in range(2)]
    comp, cs = torch.cuda.current_stream(), torch.cuda.Stream()
    h2d = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    outs = [(torch.empty_like(pos_h).pin_memory(), torch.empty_like(vel_h).pin_memory(),
             torch.empty(4, dtype=torch.float64).pin_memory()) for _ in range(2)]
    jobs, results = 5, []

    def copy_in(j):
        s = sts[j % 2]
        with torch.cuda.stream(cs):
            s.pos[s.c.cur].copy_(pos_h, non_blocking=True)
            s.vel[s.c.cur].copy_(vel_h, non_blocking=True)
            h2d[j % 2].record(cs)

    copy_in(0)
    for j in range(jobs):
        if j + 1 < jobs:
            copy_in(j + 1)
        s = sts[j % 2]
        comp.wait_event(h2d[j % 2])
        D.dcm_step_init(ctx, s, comp)
        D.dcm_step(ctx, s, 0.005, 10, comp)
        done[j % 2].record(comp)
        cs.wait_event(done[j % 2])
        po, vo, to = outs[j % 2]
        with torch.cuda.stream(cs):
            po.copy_(s.pos[s.c.cur], non_blocking=True)
            vo.copy_(s.vel[s.c.cur], non_blocking=True)
            to.copy_(s.thermo, non_blocking=True)
        if j >= 1:  # the previous job's copies out, read once they landed
            cs.synchronize()
            results.append(tuple(x.clone() for x in outs[(j - 1) % 2]))
    torch.cuda.synchronize()
    results.append(tuple(x.clone() for x in outs[(jobs - 1) % 2]))
    assert D.dcm_status(ctx) == D.DCM_OK
    assert len(results) == jobs
    for po, vo, to in results:
        assert torch.equal(po, rp) and torch.equal(vo, rv) and torch.equal(to, rt)


def run_gpu_steps_list(D, slab, P, nsteps, skin, K=10, dt=0.005, rc_max=5.5, lx=0.0, newton3=0):
    ctx = make_ctx(D, slab.box, slab.n, P, recompute_every=K, skin=skin, rc_max=rc_max, lx=lx, newton3=newton3)
    real = real_of(D, P)
    st = D.State(ctx, pos4_of(D, slab.pos, None, P), D.to_real4(torch.from_numpy(slab.vel), None, real))
    D.dcm_step_init(ctx, st)
    out = [st.thermo.cpu().numpy().copy()]
    for _ in range(nsteps):
        D.dcm_step(ctx, st, dt, 1)
        out.append(st.thermo.cpu().numpy().copy())
    assert D.dcm_status(ctx) == D.DCM_OK
    return ctx, st, np.array(out)


@pytest.mark.parametrize("lx,newton3", [(0.0, 0), (0.75, 0), (0.0, 1), (0.75, 1)])
def test_step_verlet_lists_fp64_matches_oracle(D, slab_1935, lx, newton3):
    # Verlet lists (Algorithm 2.2) with skin: same trajectory as the oracle's
    # cell-list steps (rebuilds on displacement and at every cutoff recomputation);
    # newton3: half lists, each pair evaluated once for both particles where
    # both cutoffs reach and for the larger-cutoff particle alone otherwise
    nsteps = 24
    ctx, st, th = run_gpu_steps_list(D, slab_1935, D.DCM_PREC_FP64, nsteps, skin=0.3, K=10, lx=lx,
                                     newton3=newton3)
    p = O.Params(box=slab_1935.box, recompute_every=10, rc_max=5.5)
    ost = O.init_state(slab_1935.pos, slab_1935.vel, p)
    for k in range(nsteps):
        ost = O.step(ost, 0.005, p)
        assert th[k + 1, 0] == pytest.approx(ost.E, rel=1e-9), k
        assert th[k + 1, 1] == pytest.approx(ost.W, rel=1e-9), k
        assert th[k + 1, 2] == pytest.approx(O.kinetic(ost.vel), rel=1e-9), k
        assert th[k + 1, 3] == ost_pairs(ost, p), k
    pos, vel, rc, ids = st.current()
    gp = np.empty((slab_1935.n, 3))
    gp[ids.cpu().numpy()] = pos.cpu().numpy()[:, :3]
    d = np.abs(np.mod(gp - ost.pos + 0.5 * np.array(slab_1935.box), slab_1935.box) - 0.5 * np.array(slab_1935.box))
    assert d.max() <= 1e-9


def ost_pairs(ost, p):
    return O.forces(ost.pos, ost.rc, p).npairs


def test_step_verlet_lists_mixed_close_to_cells(D, slab_1935):
    _, st_l, th_l = run_gpu_steps_list(D, slab_1935, D.DCM_PREC_MIXED, 12, skin=0.4, K=5)
    ctx = make_ctx(D, slab_1935.box, slab_1935.n, D.DCM_PREC_MIXED, recompute_every=5, rc_max=5.5)
    st = D.State(ctx, pos4_of(D, slab_1935.pos, None, D.DCM_PREC_MIXED),
                 D.to_real4(torch.from_numpy(slab_1935.vel), None, torch.float32))
    D.dcm_step_init(ctx, st)
    for _ in range(12):
        D.dcm_step(ctx, st, 0.005, 1)
    assert D.dcm_status(ctx) == D.DCM_OK
    th_c = st.thermo.cpu().numpy()
    assert th_l[-1, 0] == pytest.approx(th_c[0], rel=1e-4)
    assert th_l[-1, 2] == pytest.approx(th_c[2], rel=1e-4)
    # forces on shared inputs: the list path's positions and cutoffs given to the oracle
    pos, vel, rc, ids = st_l.current()
    pw = np.mod(pos.cpu().numpy()[:, :3].astype(np.float64), slab_1935.box)
    ref = O.forces_cells(pw, rc.cpu().numpy().astype(np.float64), slab_1935.box, 1.5)
    Fg = st_l.force.cpu().numpy().astype(np.float64)
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
    assert abs(th_l[-1, 0] - ref.E) <= EW_TOL * abs(ref.E)


@pytest.mark.parametrize("newton3", [0, 1])
def test_step_verlet_lists_mixed_medium_box(D, newton3):
    """Lists on a box where most particles have only same-image neighbours (the
    packed two-pairs-per-iteration loop) and the boundary ones image entries:
    forces after a few steps against the oracle on the same positions (full
    lists, and half lists with Newton's third law)."""
    spec = synth.SlabSpec(box=(36.0, 36.0, 144.0), wave_amp=1.0, seed=5, name="medium")
    slab = synth.make_slab(spec)
    ctx, st, th = run_gpu_steps_list(D, slab, D.DCM_PREC_MIXED, 7, skin=0.5, K=5, rc_max=6.0, newton3=newton3)
    pos, vel, rc, ids = st.current()
    pw = np.mod(pos.cpu().numpy()[:, :3].astype(np.float64), slab.box)
    ref = O.forces_cells(pw, rc.cpu().numpy().astype(np.float64), slab.box, 1.5)
    Fg = st.force.cpu().numpy().astype(np.float64)
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
    assert abs(Fg[:, 3] - ref.e).max() <= 1e-5 * np.abs(ref.e).max()
    assert abs(th[-1, 0] - ref.E) <= EW_TOL * abs(ref.E)
    assert abs(th[-1, 1] - ref.W) <= EW_TOL * abs(ref.W)
    assert abs(int(th[-1, 3]) - ref.npairs) <= near_cutoff_pairs(pw, rc.cpu().numpy().astype(np.float64), slab.box)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_step_lists_batched_call_equals_single_calls(D, slab_1935, prec):
    # Verlet-list path: one call of 12 steps == 12 calls of one step, bit for bit
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    ctx1, st1, th1 = run_gpu_steps_list(D, slab_1935, P, 12, skin=0.4, K=5)
    ctx2 = make_ctx(D, slab_1935.box, slab_1935.n, P, recompute_every=5, skin=0.4, rc_max=5.5)
    st2 = D.State(ctx2, pos4_of(D, slab_1935.pos, None, P),
                  D.to_real4(torch.from_numpy(slab_1935.vel), None, real_of(D, P)))
    D.dcm_step_init(ctx2, st2)
    D.dcm_step(ctx2, st2, 0.005, 12)
    assert D.dcm_status(ctx2) == D.DCM_OK
    assert np.array_equal(th1[-1], st2.thermo.cpu().numpy())
    assert torch.equal(st1.current()[0], st2.current()[0]) and torch.equal(st1.current()[1], st2.current()[1])


@pytest.mark.parametrize("newton3", [0, 1])
def test_newton3_two_types_asymmetric_cutoffs(D, newton3):
    """Two types, shifted energy and cutoffs spread over [3, 6] (most pairs
    within one cutoff only): the list path's forces, e_i, E, W and pair count
    against the oracle in FP64 after its initial evaluation, for full lists
    and for half lists (where a pair within both cutoffs is evaluated once and
    scattered, one within one cutoff goes to that particle alone)."""
    spec = synth.named("slab_256k_2types")
    spec.box = (18.0, 18.0, 72.0)
    slab = synth.make_slab(spec)
    n = slab.n
    P = D.DCM_PREC_FP64
    ctx = make_ctx(D, slab.box, n, P, skin=0.4, rc_max=6.0, ntypes=2, eps=(1.0, 0.8), sigma=(1.0, 1.1),
                   shift_energy=1, newton3=newton3, recompute_every=1000)
    st = D.State(ctx, pos4_of(D, slab.pos, slab.types, P), torch.zeros((n, 4), dtype=torch.float64, device="cuda"))
    D.dcm_step_init(ctx, st)
    assert D.dcm_status(ctx) == D.DCM_OK
    pos, vel, rc, ids = st.current()
    p = pos.cpu().numpy()
    rcn = rc.cpu().numpy()
    assert (rcn > 3.0).sum() > 0.2 * n   # many cutoffs above rc_min: asymmetric pairs abound
    ref = O.forces_cells(p[:, :3], rcn, slab.box, 1.5, p[:, 3].astype(np.int32), (1.0, 0.8), (1.0, 1.1), True)
    F = st.force.cpu().numpy()
    assert np.abs(F[:, :3] - ref.F).max() <= FP64_TOL * np.abs(ref.F).max()
    assert np.abs(F[:, 3] - ref.e).max() <= FP64_TOL * np.abs(ref.e).max()
    th = st.thermo.cpu().numpy()
    assert th[0] == pytest.approx(ref.E, rel=FP64_TOL) and th[1] == pytest.approx(ref.W, rel=FP64_TOL)
    assert int(th[3]) == ref.npairs


def test_newton3_needs_lists(D):
    rc, msg = D.dcm_validate_params(D.make_params((12.0, 12.0, 48.0), rc_max=5.5, newton3=1))
    assert rc == D.DCM_ERR_INVALID_ARG and "newton3" in msg
    rc, _ = D.dcm_validate_params(D.make_params((12.0, 12.0, 48.0), rc_max=5.5, skin=0.4, newton3=1))
    assert rc == D.DCM_OK


def test_skin_validation(D):
    p = D.make_params((12.0, 12.0, 48.0), skin=0.5)   # rc_max 6 + 0.5 > 12 / 2
    rc, msg = D.dcm_validate_params(p)
    assert rc == D.DCM_ERR_BOX and "skin" in msg


# ----------------------------------------------------------- full-size sample
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_error_report_per_result(D, slab_1935, prec):
    """The error of each result of the path against the FP64 oracle on the
    1,935-particle slab, stage by stage on the same inputs (printed with an
    ERR prefix, and held to the tolerances): distances, cutoffs, forces,
    per-particle energies, total energy, virial and the accepted pairs."""
    slab = slab_1935
    n = slab.n
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    real = real_of(D, P)
    ctx = make_ctx(D, slab.box, n, P)
    pos4 = pos4_of(D, slab.pos, None, P)
    cell, start, perm, ps = gpu_bin(D, ctx, pos4)
    oc, ocount, ostart, operm = O.bin_particles(slab.pos, slab.box, 1.5)
    assert np.array_equal(start, ostart) and np.array_equal(perm, operm)
    bc, g, T, s_, iface = gpu_detect(D, ctx, pos4)
    nh = O.grid_dims(slab.box, 1.5)
    og, oT, os_, oif = O.detect_interface(ocount, nh, 2)
    assert T == oT and np.array_equal(iface.cpu().numpy(), oif)
    Dg = torch.empty(ctx.nbox, dtype=real, device="cuda")
    D.dcm_distance(ctx, s_, iface, Dg)
    Do, _ = O.cfsm(os_, oif, nh, 1.5, 6.0)
    Dgn = Dg.cpu().numpy().astype(np.float64)
    fin = np.isfinite(Do)
    d_err = float(np.max(np.abs(Dgn[fin] - Do[fin]) / np.maximum(np.abs(Do[fin]), 1.5)))
    rc = torch.empty(n, dtype=real, device="cuda")
    D.dcm_cutoffs(ctx, n, ps, Dg, rc)
    spos = slab.pos[operm].astype(np.float64)
    _, orc = O.cutoffs(spos, Do, nh, 1.5, 6.0, 3.0, 6.0, 3.0)
    rcn = rc.cpu().numpy().astype(np.float64)
    rc_err = float(np.abs(rcn - orc).max())
    F = torch.empty_like(ps)
    tot = torch.zeros(3, dtype=torch.float64, device="cuda")
    D.dcm_forces(ctx, n, ps, rc, torch.from_numpy(start).cuda(), F, tot)
    torch.cuda.synchronize()
    ref = O.forces_cells(spos, rcn, slab.box, 1.5)
    Fg = F.cpu().numpy().astype(np.float64)
    tot = tot.cpu().numpy()
    f_err = rms_rel(Fg[:, :3], ref.F)
    e_err = float(np.abs(Fg[:, 3] - ref.e).max() / np.abs(ref.e).max())
    E_err = abs(tot[0] - ref.E) / abs(ref.E)
    W_err = abs(tot[1] - ref.W) / abs(ref.W)
    dp = int(tot[2]) - ref.npairs
    print(f"ERR slab_1935 {prec}: distances {d_err:.3g} (of max(D, h)), cutoffs {rc_err:.3g} (abs), "
          f"forces {f_err:.3g} (rms-rel), e_i {e_err:.3g} (of max |e_i|), E {E_err:.3g}, W {W_err:.3g} (rel), "
          f"pairs {dp:+d} of {ref.npairs}")
    if prec == "mixed":
        assert d_err <= D_TOL and rc_err <= RC_TOL and f_err <= F_RMS_TOL and e_err <= 1e-5
        assert E_err <= EW_TOL and W_err <= EW_TOL
        assert abs(dp) <= near_cutoff_pairs(spos, rcn, slab.box)
    else:
        assert max(d_err, rc_err, f_err, e_err, E_err, W_err) <= FP64_TOL and dp == 0


@pytest.fixture(scope="module")
def slab_16m():
    return synth.make_slab(synth.named("slab_16m"))


def test_full_size_sampled(D, slab_16m):
    """The 15.5M-particle workload in the configuration the benchmark times:
    whole-grid stages compared in full, forces on a sample of particles."""
    slab = slab_16m
    n = slab.n
    ctx = make_ctx(D, slab.box, n)
    pos4 = pos4_of(D, slab.pos, None, D.DCM_PREC_MIXED)
    cell, start, perm, ps = gpu_bin(D, ctx, pos4)
    oc, ocount, ostart, operm = O.bin_particles(slab.pos, slab.box, 1.5)
    assert np.array_equal(start, ostart) and np.array_equal(perm, operm)
    bc, g, T, s, iface = gpu_detect(D, ctx, pos4)
    nh = O.grid_dims(slab.box, 1.5)
    og, oT, os_, oif = O.detect_interface(ocount, nh, 2)
    assert T == oT and np.array_equal(g, og) and np.array_equal(iface.cpu().numpy(), oif)
    Dg = torch.empty(ctx.nbox, dtype=torch.float32, device="cuda")
    D.dcm_distance(ctx, s, iface, Dg)
    Do, _ = O.cfsm(os_, oif, nh, 1.5, 6.0)
    Dgn = Dg.cpu().numpy().astype(np.float64)
    assert_distances(Dgn, Do, 6.0, D_TOL)
    rc = torch.empty(n, dtype=torch.float32, device="cuda")
    D.dcm_cutoffs(ctx, n, ps, Dg, rc)
    _, orc = O.cutoffs(slab.pos[operm], Do, nh, 1.5, 6.0, 3.0, 6.0, 3.0)
    rcn = rc.cpu().numpy().astype(np.float64)
    fin = np.isfinite(Do)
    print(f"ERR slab_16m: distances max {np.max(np.abs(Dgn[fin] - Do[fin]) / np.maximum(np.abs(Do[fin]), 1.5)):.3g} "
          f"(of max(D, h)), cutoffs max abs {np.abs(rcn - orc).max():.3g}")
    assert np.abs(rcn - orc).max() <= RC_TOL
    rng = np.random.default_rng(7)
    # sample: random particles plus all of a few interface-region cells
    idx = np.unique(np.concatenate([rng.choice(n, 3000, replace=False),
                                    np.flatnonzero((rcn > 3.0) & (rcn < 6.0))[:1000]]))
    spos = slab.pos[operm].astype(np.float64)
    Fo, eo, wo, po = O.forces_subset(spos, rcn, slab.box, 1.5, idx, nthreads=8)
    totals = []
    for kernel, acc in ((0, 0), (1, 1), (1, 3), (1, 6), (3, 1), (3, 2), (3, 3), (3, 4), (3, 5), (3, 6)):
        # both cell-list kernels and the accumulation forms on the same sorted input
        kctx = make_ctx(D, slab.box, n, force_kernel=kernel, accumulation=acc)
        F = torch.empty_like(ps)
        tot = torch.zeros(3, dtype=torch.float64, device="cuda")
        D.dcm_forces(kctx, n, ps, rc, torch.from_numpy(start).cuda(), F, tot)
        torch.cuda.synchronize()
        Fs = F.cpu().numpy().astype(np.float64)[idx]
        print(f"ERR slab_16m kernel {kernel} acc {D.ACC_NAMES[D.dcm_accumulation(kctx)]}: forces rms-rel "
              f"{rms_rel(Fs[:, :3], Fo):.3g} on {len(idx)} sampled particles, e_i max "
              f"{np.abs(Fs[:, 3] - eo).max() / np.abs(eo).max():.3g} (of max |e_i|)")
        assert rms_rel(Fs[:, :3], Fo) <= F_RMS_TOL
        assert np.abs(Fs[:, 3] - eo).max() <= 1e-5 * np.abs(eo).max()
        tot = tot.cpu().numpy()
        assert tot[0] != 0.0 and np.isfinite(tot).all()
        totals.append(tot)
        del F, kctx
    # the kernels accept the same pairs up to cutoff ties and agree on the totals
    for t in totals[1:]:
        assert abs(t[2] - totals[0][2]) <= 1e-6 * totals[0][2]
        assert abs(t[0] - totals[0][0]) <= EW_TOL * abs(totals[0][0])
        assert abs(t[1] - totals[0][1]) <= EW_TOL * abs(totals[0][1])


def test_full_size_energy_virial(D, slab_16m):
    """E and W of the 15.5M-particle workload in the configuration the
    benchmark times (cells 0.5 x 1.5 x 1.5, the packed kernel) against the
    oracle's cell-list sums over ALL particles, on the same sorted positions
    and cutoffs (Section 2.4, Alg. 2.3: e_i is half the accepted pairs' U):
    E and W within 1e-7 relative in every per-particle accumulation form, the
    accepted-pair count equal up to pairs at r = rc_i within rounding (at most
    1e-6 of the pairs)."""
    import os
    slab = slab_16m
    n = slab.n
    ctx = make_ctx(D, slab.box, n, lx=0.5)
    pos4 = pos4_of(D, slab.pos, None, D.DCM_PREC_MIXED)
    cell, start, perm, ps = gpu_bin(D, ctx, pos4)
    bc, g, T, s, iface = gpu_detect(D, ctx, pos4)
    Dg = torch.empty(ctx.nbox, dtype=torch.float32, device="cuda")
    D.dcm_distance(ctx, s, iface, Dg)
    rc = torch.empty(n, dtype=torch.float32, device="cuda")
    D.dcm_cutoffs(ctx, n, ps, Dg, rc)
    starts = torch.from_numpy(start).cuda()
    torch.cuda.synchronize()
    spos = ps.cpu().numpy()[:, :3].astype(np.float64)
    rcn = rc.cpu().numpy().astype(np.float64)
    ref = O.forces_cells(spos, rcn, slab.box, 1.5, nthreads=os.cpu_count() or 1)
    worst = 0.0
    for acc in (0, 1, 2, 3, 4, 5, 6, 7):
        kctx = make_ctx(D, slab.box, n, lx=0.5, accumulation=acc)
        F = torch.empty_like(ps)
        tot = torch.zeros(3, dtype=torch.float64, device="cuda")
        D.dcm_forces(kctx, n, ps, rc, starts, F, tot)
        tot = tot.cpu().numpy()
        eE, eW = abs(tot[0] - ref.E) / abs(ref.E), abs(tot[1] - ref.W) / abs(ref.W)
        dp = int(tot[2]) - ref.npairs
        print(f"ERR slab_16m E W vs oracle (all {n} particles, acc {D.ACC_NAMES[D.dcm_accumulation(kctx)]}): "
              f"E {eE:.3g} W {eW:.3g} (rel), pairs {dp:+d} of {ref.npairs}")
        assert eE <= EW_TOL and eW <= EW_TOL
        assert abs(dp) <= 1e-6 * ref.npairs
        worst = max(worst, eE, eW)
        del F, kctx
    assert worst > 0.0  # the comparison saw FP32 pair arithmetic, not a copy


# ------------------------------------------------- curved interface (cylinder)
@pytest.fixture(scope="module")
def cyl_small():
    return synth.make_slab(synth.named("cylinder_2393"))


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_cylinder_pipeline(D, cyl_small, prec):
    """A liquid cylinder in vapor (a curved interface, Fig. 5b): detection
    bit-exact, distances, cutoffs and forces against the oracle."""
    slab = cyl_small
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    ctx = make_ctx(D, slab.box, slab.n, P)
    pos4 = pos4_of(D, slab.pos, None, P)
    bc, g, T, s, iface = gpu_detect(D, ctx, pos4)
    nh = O.grid_dims(slab.box, 1.5)
    _, ocount, _, _ = O.bin_particles(slab.pos, slab.box, 1.5)
    og, oT, os_, oif = O.detect_interface(ocount, nh, 2)
    assert np.array_equal(bc, ocount) and np.array_equal(g, og) and T == oT
    assert np.array_equal(s.cpu().numpy(), os_) and np.array_equal(iface.cpu().numpy(), oif)
    assert oif.sum() > 0
    Dg = torch.empty(ctx.nbox, dtype=real_of(D, P), device="cuda")
    D.dcm_distance(ctx, s, iface, Dg)
    Dj, _ = O.distance_jacobi(os_, oif, nh, 1.5, 6.0)
    assert_distances(Dg.cpu().numpy().astype(np.float64), Dj, 6.0, D_TOL if prec == "mixed" else FP64_TOL)
    rc = torch.empty(slab.n, dtype=real_of(D, P), device="cuda")
    D.dcm_cutoffs(ctx, slab.n, pos4, Dg, rc)
    a = O.assign_cutoffs(slab.pos, O.Params(box=slab.box))
    tol = RC_TOL if prec == "mixed" else FP64_TOL * 6
    assert np.abs(rc.cpu().numpy().astype(np.float64) - a["rc"]).max() <= tol
    Fg, tot, ref, rc_in = forces_case(D, slab, prec, a["rc"])
    if prec == "mixed":
        assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
        assert abs(tot[0] - ref.E) <= EW_TOL * abs(ref.E)
    else:
        assert np.abs(Fg[:, :3] - ref.F).max() <= FP64_TOL * np.abs(ref.F).max()
        assert int(tot[2]) == ref.npairs


def test_cylinder_299k_step_on_shared_inputs(D):
    """dcm_step_init on the 299k-particle cylinder (mixed): the oracle
    recomputes cutoffs and forces at the GPU's own sorted positions."""
    slab = synth.make_slab(synth.named("cylinder_299k"))
    ctx = make_ctx(D, slab.box, slab.n, D.DCM_PREC_MIXED, recompute_every=10)
    st = D.State(ctx, pos4_of(D, slab.pos, None, D.DCM_PREC_MIXED),
                 D.to_real4(torch.from_numpy(slab.vel), None, torch.float32))
    D.dcm_step_init(ctx, st)
    th = st.thermo.cpu().numpy()
    pos, vel, rc, ids = st.current()
    pos = pos.cpu().numpy().astype(np.float64)[:, :3]
    rcn = rc.cpu().numpy().astype(np.float64)
    a = O.assign_cutoffs(pos, O.Params(box=slab.box))
    assert np.abs(rcn - a["rc"]).max() <= RC_TOL
    ref = O.forces_cells(pos, rcn, slab.box, 1.5)
    Fg = st.force.cpu().numpy().astype(np.float64)
    assert rms_rel(Fg[:, :3], ref.F) <= F_RMS_TOL
    assert abs(th[0] - ref.E) <= EW_TOL * abs(ref.E)
    assert abs(th[1] - ref.W) <= EW_TOL * abs(ref.W)
    assert abs(int(th[3]) - ref.npairs) <= near_cutoff_pairs(pos, rcn, slab.box)
    # the curved front takes more sweeps than a slab (the oracle's Jacobi:
    # 75 on this grid); the step's sweeps run to convergence
    assert D.dcm_status(ctx) == D.DCM_OK


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_step_sweeps_equal_the_host_checked_distance(D, prec):
    """The cutoffs of dcm_step_init (all distance sweeps in one cooperative
    launch, no host check) equal, bit for bit, those of the stage calls with
    dcm_distance (one launch per sweep, host convergence check) on the same
    sorted positions; the cylinder's curved front needs about 75 sweeps."""
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    real = real_of(D, P)
    slab = synth.make_slab(synth.named("cylinder_299k"))
    ctx = make_ctx(D, slab.box, slab.n, P, recompute_every=10)
    st = D.State(ctx, pos4_of(D, slab.pos, None, P), D.to_real4(torch.from_numpy(slab.vel), None, real))
    D.dcm_step_init(ctx, st)
    assert D.dcm_status(ctx) == D.DCM_OK
    pos, _, rc, _ = st.current()
    _, _, _, s, iface = gpu_detect(D, ctx, pos)
    Dg = torch.empty(ctx.nbox, dtype=real, device="cuda")
    iters = torch.zeros(1, dtype=torch.int32, device="cuda")
    D.dcm_distance(ctx, s, iface, Dg, iters)
    assert int(iters.item()) > 40
    rc2 = torch.empty_like(rc)
    D.dcm_cutoffs(ctx, slab.n, pos, Dg, rc2)
    torch.cuda.synchronize()
    assert torch.equal(rc, rc2)


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("skin", [0.0, 0.5])
def test_empty_system_steps(D, prec, skin):
    """N = 0: every stage runs on empty arrays, the totals are zero."""
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    real = real_of(D, P)
    ctx = make_ctx(D, (12.0, 12.0, 48.0), 8, P, skin=skin, rc_max=5.5)
    st = D.State(ctx, torch.empty((0, 4), dtype=real, device="cuda"), torch.empty((0, 4), dtype=real, device="cuda"))
    D.dcm_step_init(ctx, st)
    D.dcm_step(ctx, st, 0.005, 3)
    assert D.dcm_status(ctx) == D.DCM_OK
    assert torch.count_nonzero(st.thermo).item() == 0


def two_particles(D, r, rc, prec="mixed"):
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    real = real_of(D, P)
    pts = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]], np.float32)
    ctx = make_ctx(D, (12.0, 12.0, 12.0), 2, P)
    cell, start, perm, ps = gpu_bin(D, ctx, pos4_of(D, pts, None, P))
    rcs = torch.tensor([rc, rc], dtype=real, device="cuda")
    F = torch.empty_like(ps)
    tot = torch.zeros(3, dtype=torch.float64, device="cuda")
    D.dcm_forces(ctx, 2, ps, rcs, torch.from_numpy(start).cuda(), F, tot)
    torch.cuda.synchronize()
    return F.cpu().numpy().astype(np.float64), tot.cpu().numpy()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_pair_rule_is_strict_at_the_cutoff(D, prec):
    """|r_ij| < rc_i: a pair exactly at rc is out, one ulp beyond rc is in."""
    F, tot = two_particles(D, 3.0, 3.0, prec)
    assert tot[2] == 0 and np.abs(F).max() == 0.0
    rc_up = float(np.nextafter(np.float32(3.0), np.float32(4.0)))
    F, tot = two_particles(D, 3.0, rc_up, prec)
    assert tot[2] == 2
    # U(3) = 4 (3^-12 - 3^-6); each particle carries half, the force is 24 (2 r^-13 - r^-7)
    u = 4.0 * (3.0 ** -12 - 3.0 ** -6)
    assert tot[0] == pytest.approx(u, rel=1e-6)
    f = 24.0 * (2 * 3.0 ** -13 - 3.0 ** -7)    # < 0: attraction
    assert F[0, 0] == pytest.approx(-f, rel=1e-6) and F[1, 0] == pytest.approx(f, rel=1e-6)
    assert F[0, 0] == pytest.approx(-F[1, 0], rel=1e-12) and np.abs(F[:, 1:3]).max() == 0.0


def test_single_particle_has_no_pairs(D):
    F, tot = two_particles(D, 6.0, 5.9)       # the other one (and its images) beyond rc
    assert tot[2] == 0 and tot[0] == 0.0 and np.abs(F).max() == 0.0


# -------------------------------------------------------------- bubble filter
def gpu_filter(D, s_np, box, min_component):
    ctx = make_ctx(D, box, 16, min_component=min_component)
    s_in = torch.from_numpy(np.ascontiguousarray(s_np, dtype=np.uint8)).cuda()
    s_out = torch.empty_like(s_in)
    iface = torch.empty_like(s_in)
    D.dcm_remove_small_components(ctx, s_in, s_out, iface)
    torch.cuda.synchronize()
    assert D.dcm_status(ctx) == D.DCM_OK
    return s_out.cpu().numpy(), iface.cpu().numpy()


def test_bubble_filter_hand_built_gpu(D):
    s = np.zeros((10, 10, 10), np.uint8)
    s[2:8] = 1
    s[4:6, 4:6, 4:6] = 0
    s[3:6, 1:4, 7:10] = 0
    s[0, 5, 5] = 1
    nh = np.array([10, 10, 10])
    so, io = gpu_filter(D, s.ravel(), (15.0, 15.0, 15.0), 10)
    ref, k = O.remove_small_components(s.ravel(), nh, 10)
    assert k == 2 and np.array_equal(so, ref) and np.array_equal(io, O.interface(ref, nh))


@pytest.mark.parametrize("seed,min_c", [(0, 3), (1, 8), (2, 40)])
def test_bubble_filter_random_volumes(D, seed, min_c):
    # noisy volumes: thousands of components of every size, long periodic ones included
    rng = np.random.default_rng(seed)
    nh = np.array([40, 36, 30])
    s = (rng.random(int(np.prod(nh))) < 0.5).astype(np.uint8)
    so, io = gpu_filter(D, s, tuple(1.5 * nh), min_c)
    ref, _ = O.remove_small_components(s, nh, min_c)
    assert np.array_equal(so, ref) and np.array_equal(io, O.interface(ref, nh))


def test_detect_with_filter_on_noisy_segmentation(D, slab_1935):
    # w = 0: the raw counts give a noisy S with small components in both phases
    ctx = make_ctx(D, slab_1935.box, slab_1935.n, smooth_w=0, min_component=6)
    bc, g, T, s, iface = gpu_detect(D, ctx, pos4_of(D, slab_1935.pos, None, D.DCM_PREC_MIXED))
    nh = O.grid_dims(slab_1935.box, 1.5)
    og, oT, os_, oif = O.detect_interface(bc, nh, 0, None, 6)
    _, _, raw, _ = O.detect_interface(bc, nh, 0)
    assert T == oT and np.array_equal(s.cpu().numpy(), os_) and np.array_equal(iface.cpu().numpy(), oif)
    assert not np.array_equal(raw, os_)     # the filter changed something here


def test_step_with_filter_fp64_matches_oracle(D, slab_1935):
    nsteps = 4
    ctx = make_ctx(D, slab_1935.box, slab_1935.n, D.DCM_PREC_FP64, recompute_every=1, smooth_w=1, min_component=5)
    st = D.State(ctx, pos4_of(D, slab_1935.pos, None, D.DCM_PREC_FP64),
                 D.to_real4(torch.from_numpy(slab_1935.vel), None, torch.float64))
    D.dcm_step_init(ctx, st)
    p = O.Params(box=slab_1935.box, recompute_every=1, smooth_w=1, min_component=5)
    ost = O.init_state(slab_1935.pos, slab_1935.vel, p)
    for k in range(nsteps):
        D.dcm_step(ctx, st, 0.005, 1)
        ost = O.step(ost, 0.005, p)
        th = st.thermo.cpu().numpy()
        assert th[0] == pytest.approx(ost.E, rel=1e-9), k
        assert th[3] == ost_pairs(ost, p), k
    assert D.dcm_status(ctx) == D.DCM_OK


def test_full_size_detection_with_filter(D, slab_16m):
    slab = slab_16m
    ctx = make_ctx(D, slab.box, slab.n, smooth_w=1, min_component=8)
    bc, g, T, s, iface = gpu_detect(D, ctx, pos4_of(D, slab.pos, None, D.DCM_PREC_MIXED))
    nh = O.grid_dims(slab.box, 1.5)
    og, oT, os_, oif = O.detect_interface(bc, nh, 1, None, 8)
    assert T == oT and np.array_equal(s.cpu().numpy(), os_) and np.array_equal(iface.cpu().numpy(), oif)
    assert D.dcm_status(ctx) == D.DCM_OK


@pytest.mark.parametrize("newton3", [0, 1])
def test_verlet_list_overflow_falls_back_to_exact_lists(D, newton3):
    """A blob at density 2.4 holds more neighbours within rc + skin than the
    list capacity bound (density 1.3): the build must detect the overflow,
    count exactly and fill again; forces then match the oracle."""
    g = np.arange(10) * 0.75 + 5.0
    blob = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(4)
    gas = rng.uniform(0, 18.0, size=(400, 3))
    far = np.abs(gas[:, None, :] - blob[None, :, :]).max(-1).min(1) > 1.5
    pts = np.concatenate([blob, gas[far]]).astype(np.float32)
    box = (18.0, 18.0, 18.0)
    n = len(pts)
    # uniform cutoff 3: bound = 1.3 x (4/3) pi 3.5^3 + 24 = 257 < ~360 neighbours in the blob
    ctx = make_ctx(D, box, n, D.DCM_PREC_FP64, skin=0.5, rc_min=3.0, rc_max=3.0, recompute_every=1000,
                   newton3=newton3)
    st = D.State(ctx, pos4_of(D, pts, None, D.DCM_PREC_FP64), torch.zeros((n, 4), dtype=torch.float64, device="cuda"))
    D.dcm_step_init(ctx, st)
    assert D.dcm_status(ctx) == D.DCM_OK
    pos, vel, rc, ids = st.current()
    p = pos.cpu().numpy()[:, :3]
    rcn = rc.cpu().numpy()
    assert (rcn == 3.0).all()
    ref = O.forces_cells(np.mod(p, box), rcn, box, 1.5)
    dc = blob - blob[555]
    assert (np.sqrt((dc * dc).sum(1)) < 3.5).sum() - 1 > int(4.18879020478639 * 3.5 ** 3 * 1.3) + 24
    F = st.force.cpu().numpy()[:, :3]
    assert np.abs(F - ref.F).max() <= FP64_TOL * np.abs(ref.F).max()
    assert st.thermo[3].item() == ref.npairs


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_forces_on_cells_in_any_order(D, slab_1935, prec):
    """dcm_forces takes any order of the particles inside a cell (callers may
    bin with their own sort): with every cell shuffled the accepted pairs and
    forces must match the oracle."""
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    real = real_of(D, P)
    box = slab_1935.box
    rc64 = O.assign_cutoffs(slab_1935.pos, O.Params(box=box))["rc"]
    rc_in = rc64.astype(np.float32).astype(np.float64) if prec == "mixed" else rc64
    cell, count, start, perm = O.bin_particles(slab_1935.pos, box, 1.5)
    rng = np.random.default_rng(2)
    perm = perm.copy()
    for c in np.flatnonzero(count > 1):
        seg = perm[start[c]:start[c + 1]]
        perm[start[c]:start[c + 1]] = seg[rng.permutation(len(seg))]
    ctx = make_ctx(D, box, slab_1935.n, P)
    ps = pos4_of(D, slab_1935.pos[perm], None, P)
    rcs = torch.from_numpy(rc_in[perm]).to(real).cuda()
    F = torch.empty_like(ps)
    tot = torch.zeros(3, dtype=torch.float64, device="cuda")
    D.dcm_forces(ctx, slab_1935.n, ps, rcs, torch.from_numpy(start).cuda(), F, tot)
    torch.cuda.synchronize()
    Fg = np.empty((slab_1935.n, 3))
    Fg[perm] = F.cpu().numpy()[:, :3]
    ref = O.forces_cells(slab_1935.pos, rc_in, box, 1.5)
    if prec == "fp64":
        assert np.abs(Fg - ref.F).max() <= FP64_TOL * np.abs(ref.F).max()
        assert int(tot[2].item()) == ref.npairs
    else:
        assert rms_rel(Fg, ref.F) <= F_RMS_TOL
        assert abs(int(tot[2].item()) - ref.npairs) <= near_cutoff_pairs(slab_1935.pos, rc_in, box)


@pytest.mark.parametrize("case", ["single_phase", "uniform_cutoff"])
def test_degenerate_pipelines(D, slab_1935, case):
    """The method's degenerate cases through dcm_step_init: a single-phase
    system has no interface, so every particle keeps rc_max; rc_min = rc_max
    is plain cutoff LJ.  Cutoffs and forces against the oracle."""
    if case == "single_phase":
        # 9 boxes per axis and a 9-wide box sum: every gray value is the total
        # count, so the 2-means threshold finds one phase and no interface
        rng = np.random.default_rng(8)
        box = (13.5, 13.5, 13.5)
        pos = rng.uniform(0, 13.5, size=(2000, 3)).astype(np.float32)
        vel = np.zeros((2000, 3), np.float32)
        kw, okw = dict(smooth_w=4), dict(smooth_w=4)
    else:
        box, pos, vel = slab_1935.box, slab_1935.pos, slab_1935.vel
        kw, okw = dict(rc_min=4.5, rc_max=4.5), dict(rc_min=4.5, rc_max=4.5)
    n = len(pos)
    ctx = make_ctx(D, box, n, D.DCM_PREC_FP64, **kw)
    st = D.State(ctx, pos4_of(D, pos, None, D.DCM_PREC_FP64), D.to_real4(torch.from_numpy(vel), None, torch.float64))
    D.dcm_step_init(ctx, st)
    assert D.dcm_status(ctx) == D.DCM_OK
    p_, v_, rc, ids = st.current()
    p_ = p_.cpu().numpy()[:, :3]
    rcn = rc.cpu().numpy()
    a = O.assign_cutoffs(p_, O.Params(box=box, **okw))
    assert np.abs(rcn - a["rc"]).max() <= 1e-12
    assert (rcn == (6.0 if case == "single_phase" else 4.5)).all()
    if case == "single_phase":
        assert a["iface"].sum() == 0
    ref = O.forces_cells(p_, rcn, box, 1.5)
    F = st.force.cpu().numpy()[:, :3]
    assert np.abs(F - ref.F).max() <= FP64_TOL * np.abs(ref.F).max()
    assert st.thermo[3].item() == ref.npairs


def test_scale_1m_mixed_against_fp64_run():
    """The 990,904-particle slab for 1,000 timesteps (cutoffs every 10) in
    the mixed form and in the FP64 form on the GPU.  The trajectories part
    ways (the dynamics is chaotic) but both integrate the same system: total
    energy, kinetic energy and the number of accepted pairs must agree to the
    level of the system's own statistical fluctuations."""
    import paper_1701_05242_gb300.dcm as D
    slab = synth.make_slab(synth.named("slab_1m"))
    th = {}
    for prec in (D.DCM_PREC_MIXED, D.DCM_PREC_FP64):
        ctx = make_ctx(D, slab.box, slab.n, prec, recompute_every=10)
        real = real_of(D, prec)
        st = D.State(ctx, pos4_of(D, slab.pos, None, prec), D.to_real4(torch.from_numpy(slab.vel), None, real))
        D.dcm_step_init(ctx, st)
        e0 = st.thermo.cpu().numpy().copy()
        for _ in range(10):
            D.dcm_step(ctx, st, 0.005, 100)
        assert D.dcm_status(ctx) == D.DCM_OK
        th[prec] = (e0, st.thermo.cpu().numpy().copy())
        del st, ctx
        torch.cuda.empty_cache()
    (a0, a1), (b0, b1) = th[D.DCM_PREC_MIXED], th[D.DCM_PREC_FP64]
    assert a0[0] == pytest.approx(b0[0], rel=1e-7)                 # same start
    # measured: total energy within 5e-5 at every 100 steps, kinetic energy
    # and pair count within 9e-4 (the fluctuations of a million particles)
    tot_a, tot_b = a1[0] + a1[2], b1[0] + b1[2]
    assert tot_a == pytest.approx(tot_b, rel=1e-4)
    assert a1[2] == pytest.approx(b1[2], rel=2e-3)                  # kinetic energy
    assert a1[3] == pytest.approx(b1[3], rel=2e-3)                  # accepted pairs
