"""dcm_distance_noalloc: the distance call for callers that cannot allocate
device memory (their memory belongs to another allocator, they run inside a
CUDA graph capture, or they are a plugin handed only device buffers).

Checked through the C ABI against dcm_distance on the same inputs, on two
calls in a row (the fixed scratch keeps the previous call's contents, so the
second call shows that everything that must start cleared is cleared).  This
file is collected last so that a stop at the first failure has run every
other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1701_05242_gb300 import synth

pytestmark = pytest.mark.gpu

D_TOL = 1e-5   # the distance tolerance of the parity tests


def _inputs(D, slab, prec):
    p = D.make_params(slab.box, n_max=slab.n, precision=prec)
    ctx = D.Context(p)
    _, count, _, _ = O.bin_particles(slab.pos, slab.box, 1.5)
    nh = O.grid_dims(slab.box, 1.5)
    _, _, s, iface = O.detect_interface(count, nh, 2)
    return p, ctx, torch.from_numpy(s).cuda(), torch.from_numpy(iface).cuda()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_noalloc_distance_matches_dcm_distance_twice(prec):
    import paper_1701_05242_gb300.dcm as D
    P = D.DCM_PREC_MIXED if prec == "mixed" else D.DCM_PREC_FP64
    real = torch.float32 if prec == "mixed" else torch.float64
    slab = synth.make_slab(synth.named("slab_1935"))
    p, ctx, s, iface = _inputs(D, slab, P)
    ref = torch.empty(ctx.nbox, dtype=real, device="cuda")
    it_ref = torch.empty(1, dtype=torch.int32, device="cuda")
    D.dcm_distance(ctx, s, iface, ref, it_ref)
    ref_h = ref.cpu().numpy().astype(np.float64)
    for call in range(2):
        out = torch.full((ctx.nbox,), -7.0, dtype=real, device="cuda")
        it = torch.full((1,), -9, dtype=torch.int32, device="cuda")
        assert D.dcm_distance_noalloc(p, s, iface, out, it) == D.DCM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        fin = np.isfinite(ref_h)
        assert np.array_equal(np.isfinite(got), fin), call
        assert np.all(np.abs(got[fin] - ref_h[fin]) <= D_TOL * np.maximum(ref_h[fin], 1.5)), call
        assert int(it.item()) == int(it_ref.item()), call


def test_noalloc_rejects_oversized_grid():
    import paper_1701_05242_gb300.dcm as D
    p = D.make_params((240.0, 240.0, 960.0), precision=D.DCM_PREC_MIXED)   # 16.4M boxes > 8 MiB scratch
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert D.dcm_distance_noalloc(p, dummy, dummy, out) == D.DCM_ERR_CAPACITY
