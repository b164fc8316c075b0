"""dcm_distance_noalloc: the distance call for callers that cannot allocate
device memory (their memory belongs to another allocator or framework, or
they are a plugin handed only device buffers).

Checked through the C ABI against dcm_distance on the same inputs, on two
calls in a row (the fixed scratch keeps the previous call's contents, so the
second call shows that everything that must start cleared is cleared): a
converged run, runs whose sweep budget ends before convergence after an odd
and an even number of sweeps (the last iterate must reach D either way, the
return code and iters = -1 must match), and a grid just under the fixed
scratch's limit next to one just over it.  This file is collected last so
that a stop at the first failure has run every other test first; it also
passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1701_05242_gb300 import synth

pytestmark = pytest.mark.gpu

D_TOL = 1e-5   # the distance tolerance of the parity tests
SCRATCH = 8 << 20   # bytes of the library's fixed scratch array


def _slab_inputs(slab):
    _, count, _, _ = O.bin_particles(slab.pos, slab.box, 1.5)
    nh = O.grid_dims(slab.box, 1.5)
    _, _, s, iface = O.detect_interface(count, nh, 2)
    return torch.from_numpy(s).cuda(), torch.from_numpy(iface).cuda()


def _reference(D, p, s, iface, real):
    """dcm_distance on a context: (return code, D, iters)."""
    ctx = D.Context(p)
    out = torch.empty(ctx.nbox, dtype=real, device="cuda")
    it = torch.full((1,), -9, dtype=torch.int32, device="cuda")
    rc = D.lib.dcm_distance(ctx.handle, D._ptr(s), D._ptr(iface), D._ptr(out), D._ptr(it), D._stream())
    torch.cuda.synchronize()
    D.dcm_status(ctx)   # clear the device status a non-converged run leaves
    return rc, out.cpu().numpy().astype(np.float64), int(it.item()), ctx.nbox


def _compare(D, p, s, iface, real, h):
    rc_ref, ref, it_ref, nbox = _reference(D, p, s, iface, real)
    fin = np.isfinite(ref)
    for call in range(2):
        out = torch.full((nbox,), -7.0, dtype=real, device="cuda")
        it = torch.full((1,), -9, dtype=torch.int32, device="cuda")
        rc = D.dcm_distance_noalloc(p, s, iface, out, it)
        torch.cuda.synchronize()
        assert rc == rc_ref, (call, rc, rc_ref)
        got = out.cpu().numpy().astype(np.float64)
        assert np.array_equal(np.isfinite(got), fin), call
        assert np.all(np.abs(got[fin] - ref[fin]) <= D_TOL * np.maximum(ref[fin], h)), call
        assert int(it.item()) == it_ref, (call, int(it.item()), it_ref)
    return rc_ref, it_ref


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_distance_matches_dcm_distance_twice(prec):
    import paper_1701_05242_gb300.dcm as D
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    real = torch.float32 if prec == "mixed" else torch.float64
    slab = synth.make_slab(synth.named("slab_1935"))
    s, iface = _slab_inputs(slab)
    p = D.make_params(slab.box, n_max=slab.n, precision=P)
    rc, it = _compare(D, p, s, iface, real, 1.5)
    assert rc == D.DCM_OK and it > 2


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("iter_max", [1, 2, 3, 4])
def test_noalloc_budget_ends_before_convergence(prec, iter_max):
    """Too few sweeps: DCM_ERR_NOT_CONVERGED, iters = -1 and the last iterate
    in D, whether that iterate sits in D or in the scratch copy (odd budget)."""
    import paper_1701_05242_gb300.dcm as D
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    real = torch.float32 if prec == "mixed" else torch.float64
    slab = synth.make_slab(synth.named("slab_1935"))
    s, iface = _slab_inputs(slab)
    p = D.make_params(slab.box, n_max=slab.n, precision=P, iter_max=iter_max)
    rc, it = _compare(D, p, s, iface, real, 1.5)
    assert rc == D.DCM_ERR_NOT_CONVERGED and it == -1


def _planar_grid(nh, lo, hi):
    """s = 1 on the boxes with lo <= z < hi (a liquid slab with two planar
    interfaces), iface from the oracle's liquid-side rule."""
    s = np.zeros(int(np.prod(nh)), dtype=np.uint8)
    z = np.arange(s.size) // (nh[0] * nh[1])
    s[(z >= lo) & (z < hi)] = 1
    iface = O.interface(s, np.asarray(nh, dtype=np.int64))
    return torch.from_numpy(s).cuda(), torch.from_numpy(iface).cuda()


def test_noalloc_grid_at_the_scratch_limit():
    """128 x 128 x 127 boxes in FP32 need 8,323,072 + 4,008 bytes of the
    8 MiB scratch and run; 128 x 128 x 129 boxes need more and are rejected
    before any launch."""
    import paper_1701_05242_gb300.dcm as D
    h = 1.5
    nh = (128, 128, 127)
    need = (4 * int(np.prod(nh)) + 255) // 256 * 256 + 4 * (1000 + 2)
    assert need <= SCRATCH
    p = D.make_params(tuple(n * h for n in nh), precision=D.DCM_PREC_MIXED)
    s, iface = _planar_grid(nh, 40, 90)
    rc, it = _compare(D, p, s, iface, torch.float32, h)
    assert rc == D.DCM_OK and it > 2
    big = (128, 128, 129)
    assert (4 * int(np.prod(big)) + 255) // 256 * 256 + 4 * (1000 + 2) > SCRATCH
    p2 = D.make_params(tuple(n * h for n in big), precision=D.DCM_PREC_MIXED)
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert D.dcm_distance_noalloc(p2, s, iface, out) == D.DCM_ERR_CAPACITY


def test_noalloc_rejects_oversized_grid():
    import paper_1701_05242_gb300.dcm as D
    p = D.make_params((240.0, 240.0, 960.0), precision=D.DCM_PREC_MIXED)   # 16.4M boxes > 8 MiB scratch
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert D.dcm_distance_noalloc(p, dummy, dummy, out) == D.DCM_ERR_CAPACITY
