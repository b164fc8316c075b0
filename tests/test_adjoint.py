"""Differentiation form: the adjoint of the force/energy map.

Loss L = sum_i |F_i|^2 + E (the two-type workload's loss), cutoffs fixed.
CPU: the oracle adjoint is pinned by central finite differences of the
oracle's own forward pass and by a dense PyTorch autograd of the same loss.
GPU: dcm_forces_backward and the autograd Function against the oracle, and
central finite differences (h = 1e-4, FP64 form).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1701_05242_gb300 import synth

EPS = (1.0, 0.8)
SIG = (1.0, 1.1)


@pytest.fixture(scope="module")
def small2():
    spec = synth.named("slab_256k_2types")
    spec.box = (12.0, 12.0, 48.0)
    slab = synth.make_slab(spec)
    rng = np.random.default_rng(9)
    rc = rng.choice([3.0, 4.0, 5.0, 6.0], slab.n)
    return slab, rc


def loss_and_forces(pos, rc, box, types, eps=EPS, sig=SIG, shift=False):
    r = O.forces_brute(pos, rc, box, types, eps, sig, shift)
    return float((r.F ** 2).sum() + r.E), r


def crosses(pos, k, rc, box, h):
    """True if moving particle k by up to h could take a pair across a cutoff."""
    d = pos[k] - pos
    d -= np.asarray(box) * np.round(d / np.asarray(box))
    r = np.sqrt((d * d).sum(1))
    r[k] = np.inf
    return bool((np.abs(r - rc[k]) < 2 * h).any() or (np.abs(r - rc) < 2 * h).any())


# ------------------------------------------------------------------ CPU pins
@pytest.mark.parametrize("shift", [False, True])
def test_oracle_adjoint_finite_differences(small2, shift):
    slab, rc = small2
    m = 500
    pos = slab.pos.astype(np.float64)[:m]
    t = slab.types[:m]
    rc = rc[:m]
    L0, r = loss_and_forces(pos, rc, slab.box, t, shift=shift)
    G, de, ds = O.adjoint(pos, rc, slab.box, 2 * r.F, 1.0, t, EPS, SIG, shift)
    h = 1e-6
    done = 0
    for k in range(m):
        if crosses(pos, k, rc, slab.box, h):
            continue
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[k, d] += h
            pm[k, d] -= h
            fd = (loss_and_forces(pp, rc, slab.box, t, shift=shift)[0] -
                  loss_and_forces(pm, rc, slab.box, t, shift=shift)[0]) / (2 * h)
            assert G[k, d] == pytest.approx(fd, rel=1e-5, abs=1e-3 * (abs(G[k]).max() + 1))
        done += 1
        if done == 4:
            break
    assert done == 4
    for a in range(2):
        for which, grad in (("eps", de), ("sig", ds)):
            e1, e2 = list(EPS), list(EPS)
            s1, s2 = list(SIG), list(SIG)
            if which == "eps":
                e1[a] += 1e-6
                e2[a] -= 1e-6
            else:
                s1[a] += 1e-6
                s2[a] -= 1e-6
            fd = (loss_and_forces(pos, rc, slab.box, t, tuple(e1), tuple(s1), shift)[0] -
                  loss_and_forces(pos, rc, slab.box, t, tuple(e2), tuple(s2), shift)[0]) / 2e-6
            assert grad[a] == pytest.approx(fd, rel=1e-6)


def test_oracle_adjoint_matches_dense_autograd(small2):
    """The same loss written as dense torch FP64 tensors (neighbour masks
    fixed at the evaluation point) and differentiated by torch.autograd."""
    slab, rc = small2
    m = 300
    pos = slab.pos.astype(np.float64)[:m]
    t = slab.types[:m]
    rcm = rc[:m]
    box = torch.tensor(slab.box, dtype=torch.float64)
    P = torch.tensor(pos, requires_grad=True)
    E_t = torch.tensor(EPS, dtype=torch.float64, requires_grad=True)
    S_t = torch.tensor(SIG, dtype=torch.float64, requires_grad=True)
    tt = torch.tensor(t, dtype=torch.long)
    d = P[:, None, :] - P[None, :, :]
    d = d - box * torch.round(d.detach() / box)
    r2 = (d * d).sum(-1)
    mask = (r2.detach() < torch.tensor(rcm)[:, None] ** 2) & ~torch.eye(m, dtype=torch.bool)
    eps_ij = torch.sqrt(E_t[tt][:, None] * E_t[tt][None, :])
    sig_ij = 0.5 * (S_t[tt][:, None] + S_t[tt][None, :])
    r2s = torch.where(mask, r2, torch.ones_like(r2))
    s6 = (sig_ij ** 2 / r2s) ** 3
    g = torch.where(mask, 24 * eps_ij * (2 * s6 * s6 - s6) / r2s, torch.zeros_like(r2))
    U = torch.where(mask, 4 * eps_ij * (s6 * s6 - s6), torch.zeros_like(r2))
    F = (g[:, :, None] * d).sum(1)
    L = (F * F).sum() + 0.5 * U.sum()
    gP, gE, gS = torch.autograd.grad(L, (P, E_t, S_t))
    r = O.forces_brute(pos, rcm, slab.box, t, EPS, SIG)
    G, de, ds = O.adjoint(pos, rcm, slab.box, 2 * r.F, 1.0, t, EPS, SIG)
    assert np.abs(G - gP.numpy()).max() <= 1e-9 * np.abs(G).max()
    assert np.allclose(de, gE.numpy(), rtol=1e-10)
    assert np.allclose(ds, gS.numpy(), rtol=1e-10)


# -------------------------------------------------------------------- GPU
def gpu_setup(D, slab, rc64, prec, shift=False, lx=0.0):
    real = torch.float32 if prec == D.DCM_PREC_MIXED else torch.float64
    p = D.make_params(slab.box, n_max=slab.n, precision=prec, ntypes=2, eps=EPS, sigma=SIG, shift_energy=int(shift),
                      lx=lx)
    ctx = D.Context(p)
    pos4 = D.to_real4(torch.from_numpy(slab.pos), torch.from_numpy(slab.types), real)
    n = slab.n
    cell = torch.empty(n, dtype=torch.int32, device="cuda")
    start = torch.empty(ctx.ncell + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    ps = torch.empty_like(pos4)
    D.dcm_bin(ctx, n, pos4, cell, start, perm, ps)
    permh = perm.cpu().numpy()
    rc_in = rc64.astype(np.float32).astype(np.float64) if prec == D.DCM_PREC_MIXED else rc64
    rcs = torch.from_numpy(rc_in[permh]).to(real).cuda()
    return ctx, ps, rcs, start, permh, rc_in


def gpu_adjoint_against_oracle(D, slab, rc, prec, lx=0.0):
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    ctx, ps, rcs, start, perm, rc_in = gpu_setup(D, slab, rc, P, lx=lx)
    n = slab.n
    F = torch.empty_like(ps)
    D.dcm_forces(ctx, n, ps, rcs, start, F)
    A = torch.zeros_like(ps)
    A[:, :3] = 2 * F[:, :3]
    G = torch.empty_like(ps)
    dpar = torch.zeros(4, dtype=torch.float64, device="cuda")
    D.dcm_forces_backward(ctx, n, ps, rcs, start, A, 1.0, G, dpar)
    torch.cuda.synchronize()
    spos = slab.pos[perm].astype(np.float64)
    st = slab.types[perm]
    r = O.forces_brute(spos, rc_in[perm], slab.box, st, EPS, SIG)
    Go, de, ds = O.adjoint(spos, rc_in[perm], slab.box, 2 * r.F, 1.0, st, EPS, SIG)
    Gg = G.cpu().numpy().astype(np.float64)[:, :3]
    err = np.sqrt(((Gg - Go) ** 2).sum() / (Go ** 2).sum())
    d = dpar.cpu().numpy()
    if prec == "mixed":
        assert err <= 1e-4
        assert np.allclose(d[:2], de, rtol=1e-4) and np.allclose(d[2:], ds, rtol=1e-4)
    else:
        assert err <= 1e-10
        assert np.allclose(d[:2], de, rtol=1e-10) and np.allclose(d[2:], ds, rtol=1e-10)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("lx", [0.0, 0.75])
def test_gpu_adjoint_matches_oracle(small2, prec, lx):
    import paper_1701_05242_gb300.dcm as D
    slab, rc = small2
    gpu_adjoint_against_oracle(D, slab, rc, prec, lx)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_gpu_adjoint_with_the_method_cutoffs(prec):
    """Cutoffs from the method itself on a slab thick enough for a bulk at
    rc_min far from both interfaces: there the reverse-pair walk is bounded
    by the blocks' largest cutoff instead of rc_max, and the gradients must
    still match the oracle's all-pairs adjoint."""
    import paper_1701_05242_gb300.dcm as D
    spec = synth.named("slab_256k_2types")
    spec.box = (13.5, 13.5, 108.0)
    slab = synth.make_slab(spec)
    rc = O.assign_cutoffs(slab.pos, O.Params(box=slab.box))["rc"]
    assert (rc <= 3.0).mean() > 0.3  # a bulk at rc_min, beyond a block of the interfaces
    gpu_adjoint_against_oracle(D, slab, rc, prec)


@pytest.mark.gpu
def test_autograd_function_and_finite_differences(small2):
    import paper_1701_05242_gb300.dcm as D
    from paper_1701_05242_gb300.autograd import lj_forces
    slab, rc = small2
    P = D.DCM_PREC_FP64
    ctx, ps, rcs, start, perm, rc_in = gpu_setup(D, slab, rc, P)
    pos = ps.clone().requires_grad_(True)
    eps = torch.tensor(EPS, dtype=torch.float64, device="cuda", requires_grad=True)
    sig = torch.tensor(SIG, dtype=torch.float64, device="cuda", requires_grad=True)
    F, E = lj_forces(pos, eps, sig, rcs, start, ctx)
    L = (F * F).sum() + E
    gp, ge, gs = torch.autograd.grad(L, (pos, eps, sig))
    spos = slab.pos[perm].astype(np.float64)
    st = slab.types[perm]
    r = O.forces_brute(spos, rc_in[perm], slab.box, st, EPS, SIG)
    Go, de, ds = O.adjoint(spos, rc_in[perm], slab.box, 2 * r.F, 1.0, st, EPS, SIG)
    assert np.abs(gp.cpu().numpy()[:, :3] - Go).max() <= 1e-9 * np.abs(Go).max()
    assert np.allclose(ge.cpu().numpy(), de, rtol=1e-10) and np.allclose(gs.cpu().numpy(), ds, rtol=1e-10)

    # central differences of the GPU FP64 forward, h = 1e-4, away from cutoffs
    def L_at(p4):
        with torch.no_grad():
            Fp, Ep = lj_forces(p4, eps, sig, rcs, start, ctx)
            return float((Fp * Fp).sum() + Ep)
    h = 1e-4
    checked = 0
    base = ps.detach()
    rch = rc_in[perm]
    for k in range(0, slab.n, 97):
        if crosses(spos, k, rch, slab.box, h):
            continue
        if (np.floor((spos[k] + h) / 1.5) != np.floor((spos[k] - h) / 1.5)).any():
            continue  # the perturbation would move k to another cell of the fixed cell list
        for d in range(3):
            pp, pm = base.clone(), base.clone()
            pp[k, d] += h
            pm[k, d] -= h
            fd = (L_at(pp) - L_at(pm)) / (2 * h)
            # rounding floor of a central difference of L: ~|L| eps / h (x20)
            floor = 20 * abs(float(L)) * 2.2e-16 / h
            assert gp[k, d].item() == pytest.approx(fd, rel=2e-4, abs=floor)
        checked += 1
        if checked == 6:
            break
    assert checked == 6


@pytest.mark.gpu
def test_adjoint_full_two_type_workload():
    """The 260,522-particle two-type workload: the mixed-precision adjoint
    against the FP64 one (itself checked against the oracle above), and the
    FP64 position gradient against central differences of the GPU FP64
    forward at a few particles."""
    import paper_1701_05242_gb300.dcm as D
    slab = synth.make_slab(synth.named("slab_256k_2types"))
    rng = np.random.default_rng(5)
    rc = rng.choice([3.0, 4.0, 5.0, 6.0], slab.n)
    out = {}
    for prec in (D.DCM_PREC_FP64, D.DCM_PREC_MIXED):
        ctx, ps, rcs, start, perm, rc_in = gpu_setup(D, slab, rc, prec)
        F = torch.empty_like(ps)
        D.dcm_forces(ctx, slab.n, ps, rcs, start, F)
        A = torch.zeros_like(ps)
        A[:, :3] = 2 * F[:, :3]
        G = torch.empty_like(ps)
        dpar = torch.zeros(4, dtype=torch.float64, device="cuda")
        D.dcm_forces_backward(ctx, slab.n, ps, rcs, start, A, 1.0, G, dpar)
        torch.cuda.synchronize()
        out[prec] = (G.cpu().numpy().astype(np.float64)[:, :3], dpar.cpu().numpy(), perm, ctx, ps, rcs, start)
    G64, d64, perm, ctx, ps, rcs, start = out[D.DCM_PREC_FP64]
    G32, d32 = out[D.DCM_PREC_MIXED][0], out[D.DCM_PREC_MIXED][1]
    assert np.array_equal(out[D.DCM_PREC_MIXED][2], perm)
    assert np.sqrt(((G32 - G64) ** 2).sum() / (G64 ** 2).sum()) <= 1e-4
    assert np.allclose(d32, d64, rtol=1e-4)

    def L_at(p4):
        F = torch.empty_like(p4)
        tot = torch.zeros(3, dtype=torch.float64, device="cuda")
        D.dcm_forces(ctx, slab.n, p4, rcs, start, F, tot)
        return float((F[:, :3] ** 2).sum() + tot[0])
    h = 1e-4
    spos = slab.pos[perm].astype(np.float64)
    rch = rcs.cpu().numpy()
    checked = 0
    for k in rng.permutation(slab.n)[:200]:
        if crosses(spos, k, rch, slab.box, h):
            continue
        if (np.floor((spos[k] + h) / 1.5) != np.floor((spos[k] - h) / 1.5)).any():
            continue
        L0 = L_at(ps)
        for d in range(3):
            pp, pm = ps.clone(), ps.clone()
            pp[k, d] += h
            pm[k, d] -= h
            fd = (L_at(pp) - L_at(pm)) / (2 * h)
            floor = 20 * abs(L0) * 2.2e-16 / h
            assert G64[k, d] == pytest.approx(fd, rel=2e-4, abs=floor)
        checked += 1
        if checked == 3:
            break
    assert checked == 3
