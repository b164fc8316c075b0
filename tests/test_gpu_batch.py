"""Batched form: independent replicas stepped together, two persistent launches
per timestep by default (or one launch per stage).

Each replica of a batch must evolve exactly as the same system stepped alone
through dcm_step (the per-particle arithmetic is the same; only the order of
the per-replica energy sums differs), a captured CUDA graph must replay the
same trajectory as direct stepping, and the FP64 batch must track the oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1701_05242_gb300 import synth

pytestmark = pytest.mark.gpu

K = 5
DT = 0.005


@pytest.fixture(scope="module")
def D():
    import paper_1701_05242_gb300.dcm as dcm
    return dcm


@pytest.fixture(scope="module")
def replicas():
    out = []
    for r, (L, rho) in enumerate([(12.0, 0.8), (13.5, 0.7), (15.0, 0.85)]):
        spec = synth.SlabSpec(box=(L, L, 4 * L), rho_l=rho, seed=r, name=f"rep{r}")
        out.append(synth.make_slab(spec))
    return out


def batch_state(D, reps, prec, lx=0.0):
    real = torch.float32 if prec == D.DCM_PREC_MIXED else torch.float64
    p = D.make_params((1, 1, 1), precision=prec, recompute_every=K, lx=lx)
    b = D.Batch(p, [s.box for s in reps], [s.n for s in reps])
    pos = np.concatenate([s.pos for s in reps])
    vel = np.concatenate([s.vel for s in reps])
    st = D.BatchState(b, D.to_real4(torch.from_numpy(pos), None, real), D.to_real4(torch.from_numpy(vel), None, real))
    return b, st


def single_run(D, slab, prec, nsteps, lx=0.0):
    real = torch.float32 if prec == D.DCM_PREC_MIXED else torch.float64
    ctx = D.Context(D.make_params(slab.box, n_max=slab.n, precision=prec, recompute_every=K, lx=lx))
    st = D.State(ctx, D.to_real4(torch.from_numpy(slab.pos), None, real), D.to_real4(torch.from_numpy(slab.vel), None, real))
    D.dcm_step_init(ctx, st)
    D.dcm_step(ctx, st, DT, nsteps)
    pos, vel, rc, ids = st.current()
    order = torch.argsort(ids.long())
    return pos[order].cpu().numpy(), st.thermo.cpu().numpy()


def by_id(st, b, r):
    pos, vel, rc, ids = st.current()
    a, e = b.offsets[r], b.offsets[r + 1]
    idr = ids[a:e].long() - a
    out = torch.empty_like(pos[a:e])
    out[idr] = pos[a:e]
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("lx", [0.0, 0.75])
def test_batch_matches_single_systems(D, replicas, prec, lx):
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    nsteps = 2 * K + 2
    b, st = batch_state(D, replicas, P, lx)
    D.dcm_batch_step_init(b, st)
    D.dcm_batch_step(b, st, DT, nsteps)
    assert D.dcm_batch_status(b) == D.DCM_OK
    th = st.thermo.cpu().numpy().reshape(-1, 4)
    for r, slab in enumerate(replicas):
        pos1, th1 = single_run(D, slab, P, nsteps, lx)
        pb = by_id(st, b, r)
        assert np.abs(pb - pos1).max() <= (1e-12 if prec == "fp64" else 1e-5)
        tol = 1e-10 if prec == "fp64" else 1e-6
        for q in range(3):
            assert th[r, q] == pytest.approx(th1[q], rel=tol, abs=1e-9)
        assert th[r, 3] == th1[3]


def test_batch_two_types_matches_single_systems(D):
    """Replicas of two types (Lorentz-Berthelot mixing, the packed typed
    loop in both paths) evolve as the same systems stepped alone."""
    reps = []
    for r, L in enumerate((12.0, 13.5)):
        spec = synth.SlabSpec(box=(L, L, 4 * L), ntypes=2, seed=10 + r, name=f"typed{r}")
        reps.append(synth.make_slab(spec))
    kw = dict(precision=D.DCM_PREC_MIXED, recompute_every=K, ntypes=2, eps=(1.0, 0.8), sigma=(1.0, 1.1))
    b = D.Batch(D.make_params((1, 1, 1), **kw), [s.box for s in reps], [s.n for s in reps])
    pos = np.concatenate([s.pos for s in reps])
    vel = np.concatenate([s.vel for s in reps])
    typ = np.concatenate([s.types for s in reps])
    st = D.BatchState(b, D.to_real4(torch.from_numpy(pos), torch.from_numpy(typ), torch.float32),
                      D.to_real4(torch.from_numpy(vel), None, torch.float32))
    nsteps = K + 2
    D.dcm_batch_step_init(b, st)
    D.dcm_batch_step(b, st, DT, nsteps)
    assert D.dcm_batch_status(b) == D.DCM_OK
    th = st.thermo.cpu().numpy().reshape(-1, 4)
    for r, slab in enumerate(reps):
        ctx = D.Context(D.make_params(slab.box, n_max=slab.n, **kw))
        assert D.dcm_force_kernel(ctx) == D.DCM_FORCE_PACKED
        s1 = D.State(ctx, D.to_real4(torch.from_numpy(slab.pos), torch.from_numpy(slab.types), torch.float32),
                     D.to_real4(torch.from_numpy(slab.vel), None, torch.float32))
        D.dcm_step_init(ctx, s1)
        D.dcm_step(ctx, s1, DT, nsteps)
        p1, _, _, ids = s1.current()
        order = torch.argsort(ids.long())
        pb = by_id(st, b, r)
        assert np.abs(pb - p1[order].cpu().numpy()).max() <= 1e-5
        t1 = s1.thermo.cpu().numpy()
        for q in range(3):
            assert th[r, q] == pytest.approx(t1[q], rel=1e-6)
    b.close()


def test_batch_graph_replay_equals_stepping(D, replicas):
    P = D.DCM_PREC_MIXED
    b1, s1 = batch_state(D, replicas, P)
    D.dcm_batch_step_init(b1, s1)
    D.dcm_batch_step(b1, s1, DT, 2 * K)
    b2, s2 = batch_state(D, replicas, P)
    D.dcm_batch_step_init(b2, s2)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    D.dcm_batch_capture(b2, s2, DT, stream)
    assert D.dcm_batch_graph_steps(b2) == (2 * K if K % 2 else K)
    reps = (2 * K) // D.dcm_batch_graph_steps(b2)
    D.dcm_batch_replay(b2, s2, reps, stream)
    stream.synchronize()
    assert s2.c.t == s1.c.t == 2 * K
    assert torch.equal(s1.current()[0], s2.current()[0])
    assert torch.equal(s1.thermo, s2.thermo)
    assert D.dcm_batch_status(b2) == D.DCM_OK


@pytest.mark.parametrize("lx", [0.0, 0.5])
def test_batch_fp64_tracks_oracle(D, replicas, lx):
    b, st = batch_state(D, replicas, D.DCM_PREC_FP64, lx)
    D.dcm_batch_step_init(b, st)
    D.dcm_batch_step(b, st, DT, 3)
    assert D.dcm_batch_status(b) == D.DCM_OK
    th = st.thermo.cpu().numpy().reshape(-1, 4)
    for r, slab in enumerate(replicas):
        p = O.Params(box=slab.box, recompute_every=K)
        o = O.init_state(slab.pos, slab.vel, p)
        for _ in range(3):
            o = O.step(o, DT, p)
        assert th[r, 0] == pytest.approx(o.E, rel=1e-9)
        assert th[r, 2] == pytest.approx(O.kinetic(o.vel), rel=1e-9)
        pb = by_id(st, b, r)
        d = np.abs(pb[:, :3] - o.pos)
        d = np.minimum(d, np.array(slab.box) - d)
        assert d.max() <= 1e-9


def test_batch_thermo_over_several_chunks(D):
    """A replica larger than one reduction chunk (4096 particles) between two
    small ones: per-replica E, W, KE and pairs equal the systems stepped alone."""
    reps = [synth.make_slab(synth.SlabSpec(box=b, seed=s, name=f"c{s}"))
            for s, b in enumerate([(12.0, 12.0, 48.0), (24.0, 24.0, 96.0), (13.5, 13.5, 54.0)])]
    assert reps[1].n > 2 * 4096
    b, st = batch_state(D, reps, D.DCM_PREC_FP64)
    D.dcm_batch_step_init(b, st)
    D.dcm_batch_step(b, st, DT, 3)
    assert D.dcm_batch_status(b) == D.DCM_OK
    th = st.thermo.cpu().numpy().reshape(-1, 4)
    for r, slab in enumerate(reps):
        _, th1 = single_run(D, slab, D.DCM_PREC_FP64, 3)
        for q in range(3):
            assert th[r, q] == pytest.approx(th1[q], rel=1e-10, abs=1e-9)
        assert th[r, 3] == th1[3]


def test_batch_rejects_bad_replica(D):
    p = D.make_params((1, 1, 1))
    with pytest.raises(D.DcmError):
        D.Batch(p, [(12.0, 12.0, 48.0), (12.0, 12.0, 47.0)], [10, 10])


# ------------------------------------------------ persistent plan (default)
def _run_plan(D, reps, P, persistent, nsteps, lx=0.0):
    b, st = batch_state(D, reps, P, lx)
    D.dcm_batch_set_persistent(b, persistent)
    D.dcm_batch_step_init(b, st)
    D.dcm_batch_launch_count(b, reset=True)
    D.dcm_batch_step(b, st, DT, nsteps)
    launches = D.dcm_batch_launch_count(b)
    assert D.dcm_batch_status(b) == D.DCM_OK
    pos, vel, rc, ids = st.current()
    out = [t.cpu().numpy() for t in (pos, vel, rc, ids, st.force)]
    return out, st.thermo.cpu().numpy().reshape(-1, 4), launches, b


@pytest.mark.parametrize("prec,lx", [("mixed", 0.0), ("mixed", 0.5), ("fp64", 0.0)])
def test_persistent_plan_equals_per_stage_plan(D, replicas, prec, lx):
    """One cooperative launch per timestep (grid barriers between the
    stages, forces from the (replica, tile) queue) steps the same trajectory
    as one launch per stage: positions, velocities, cutoffs, ids and forces
    bit for bit (the same per-element code, the binning's order fixed by the
    stable sort), per-replica totals to rounding (their block sums differ in
    width).  The persistent plan launches exactly two kernels per timestep."""
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    nsteps = 2 * K + 3   # two recomputations, an odd step count (buffers end on the other side)
    a, tha, la, _ = _run_plan(D, replicas, P, True, nsteps, lx)
    s, ths, ls, _ = _run_plan(D, replicas, P, False, nsteps, lx)
    for x, y in zip(a, s):
        assert np.array_equal(x, y)
    assert np.allclose(tha, ths, rtol=1e-12, atol=1e-9)
    assert la == 2 * nsteps
    assert ls > 5 * nsteps


@pytest.mark.parametrize("persistent", [True, False])
def test_batch_call_of_several_steps_equals_single_steps(D, replicas, persistent):
    """One call of several timesteps (forces only before its last timestep:
    no energy, virial or thermo stages) leaves the state, the forces with
    their per-particle energies, and the per-replica thermo bit-identical to
    the same timesteps taken one call each (energy and thermo every time)."""
    P = D.DCM_PREC_MIXED
    nsteps = K + 2
    a, tha, _, _ = _run_plan(D, replicas, P, persistent, nsteps)
    b, st = batch_state(D, replicas, P)
    D.dcm_batch_set_persistent(b, persistent)
    D.dcm_batch_step_init(b, st)
    for _ in range(nsteps):
        D.dcm_batch_step(b, st, DT, 1)
    assert D.dcm_batch_status(b) == D.DCM_OK
    pos, vel, rc, ids = st.current()
    for x, y in zip(a, [t.cpu().numpy() for t in (pos, vel, rc, ids, st.force)]):
        assert np.array_equal(x, y)
    assert np.array_equal(tha, st.thermo.cpu().numpy().reshape(-1, 4))


def test_persistent_plan_two_types_and_accumulation_forms(D):
    """Two types on the packed typed loop, each batched accumulation form."""
    reps = []
    for r, L in enumerate((12.0, 13.5)):
        reps.append(synth.make_slab(synth.SlabSpec(box=(L, L, 4 * L), ntypes=2, seed=20 + r, name=f"pt{r}")))
    pos = np.concatenate([s.pos for s in reps])
    vel = np.concatenate([s.vel for s in reps])
    typ = np.concatenate([s.types for s in reps])
    res, init = {}, {}
    for acc in (D.DCM_ACC_FP32, D.DCM_ACC_PLANE_KAHAN, D.DCM_ACC_PLANE_FP64):
        for persistent in (True, False):
            kw = dict(precision=D.DCM_PREC_MIXED, recompute_every=K, ntypes=2, eps=(1.0, 0.8), sigma=(1.0, 1.1),
                      accumulation=acc)
            b = D.Batch(D.make_params((1, 1, 1), **kw), [s.box for s in reps], [s.n for s in reps])
            D.dcm_batch_set_persistent(b, persistent)
            st = D.BatchState(b, D.to_real4(torch.from_numpy(pos), torch.from_numpy(typ), torch.float32),
                              D.to_real4(torch.from_numpy(vel), None, torch.float32))
            D.dcm_batch_step_init(b, st)
            init[acc, persistent] = st.thermo.cpu().numpy().copy()
            D.dcm_batch_step(b, st, DT, K + 1)
            assert D.dcm_batch_status(b) == D.DCM_OK
            res[acc, persistent] = (st.current()[0].cpu().numpy(), st.thermo.cpu().numpy())
            b.close()
        assert np.array_equal(res[acc, True][0], res[acc, False][0])
        assert np.allclose(res[acc, True][1], res[acc, False][1], rtol=1e-12)
    # on the same positions the forms differ only in how the same pair terms
    # are summed (the trajectories of the steps part ways: the dynamics from
    # the random placement are chaotic)
    e = [init[acc, True].reshape(-1, 4) for acc in (1, 7, 6)]
    for q in (0, 1):
        assert np.allclose(e[0][:, q], e[1][:, q], rtol=1e-7) and np.allclose(e[1][:, q], e[2][:, q], rtol=1e-7)
    assert np.array_equal(e[0][:, 3], e[1][:, 3]) and np.array_equal(e[1][:, 3], e[2][:, 3])


def test_persistent_plan_graph_replay(D, replicas):
    """The persistent step captured in a CUDA graph (two kernels per timestep
    in the graph) replays the trajectory of direct stepping bit for bit."""
    P = D.DCM_PREC_MIXED
    b1, s1 = batch_state(D, replicas, P)
    D.dcm_batch_step_init(b1, s1)
    D.dcm_batch_step(b1, s1, DT, 2 * K)
    b2, s2 = batch_state(D, replicas, P)
    D.dcm_batch_step_init(b2, s2)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    D.dcm_batch_capture(b2, s2, DT, stream)
    per = D.dcm_batch_graph_steps(b2)
    D.dcm_batch_launch_count(b2, reset=True)
    D.dcm_batch_replay(b2, s2, (2 * K) // per, stream)
    stream.synchronize()
    assert D.dcm_batch_launch_count(b2) == 4 * K
    assert torch.equal(s1.current()[0], s2.current()[0])
    assert torch.equal(s1.thermo, s2.thermo)
    assert D.dcm_batch_status(b2) == D.DCM_OK


def test_persistent_barrier_wait_runs_out(D, replicas):
    """The bounded grid barrier: waiting for a block that does not exist, every
    block gives up after the budget (50 ms) with DCM_ERR_TIMEOUT and returns;
    with nothing missing it passes.  The batch steps normally afterwards."""
    import time
    b, st = batch_state(D, replicas, D.DCM_PREC_MIXED)
    t0 = time.perf_counter()
    assert D.dcm_batch_barrier_selftest(b, 1, 50_000_000) == D.DCM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 20.0
    assert D.dcm_batch_barrier_selftest(b, 0, 50_000_000) == D.DCM_OK
    D.dcm_batch_step_init(b, st)
    D.dcm_batch_step(b, st, DT, 2)
    assert D.dcm_batch_status(b) == D.DCM_OK
    assert np.isfinite(st.thermo.cpu().numpy()).all()


def test_persistent_step_with_an_exhausted_wait_budget(D, replicas):
    """A wait budget of 1 microsecond, far below a stage's duration: the
    launch's barriers run out, every block leaves, and the status reports
    DCM_ERR_TIMEOUT instead of a hang; with the budget restored the batch
    steps again and matches a fresh run."""
    P = D.DCM_PREC_MIXED
    b, st = batch_state(D, replicas, P)
    D.dcm_batch_step_init(b, st)
    assert D.dcm_batch_status(b) == D.DCM_OK
    D.dcm_batch_set_wait_budget(b, 1000)
    D.dcm_batch_step(b, st, DT, 1)
    assert D.dcm_batch_status(b) == D.DCM_ERR_TIMEOUT
    D.dcm_batch_set_wait_budget(b, 2_000_000_000)
    b2, s2 = batch_state(D, replicas, P)
    for bb, ss in ((b, st), (b2, s2)):
        fresh = batch_state(D, replicas, P)[1]
        for k in range(2):
            ss.pos[k].copy_(fresh.pos[k])
            ss.vel[k].copy_(fresh.vel[k])
            ss.id[k].copy_(fresh.id[k])
        ss.c.cur = 0
        D.dcm_batch_step_init(bb, ss)
        D.dcm_batch_step(bb, ss, DT, 3)
        assert D.dcm_batch_status(bb) == D.DCM_OK
    assert torch.equal(st.current()[0], s2.current()[0])
