"""Autotuner for the batched form: picks the force-cell edges (l, and lx
along the rows) and the launch plan with its work size by timing a few steps
of every candidate on the actual replicas (CUDA events on the stepping
stream).

Candidates: (l, lx) in {(1.5, 1.5), (1.5, 0.75), (1.5, 0.5), (1.0, 1.0),
(0.75, 0.75)} where both divide every replica box (h = 1.5 stays the
density-grid edge), crossed with the persistent plan at force-queue tiles of
{32, 64, 128} particles and the per-stage plan at force blocks of {64, 128,
256} threads.
"""
from __future__ import annotations

import torch

from . import dcm as D

EDGES = ((1.5, 1.5), (1.5, 0.75), (1.5, 0.5), (1.0, 1.0), (0.75, 0.75))
PLANS = (("persistent", 32), ("persistent", 64), ("persistent", 128),
         ("stages", 64), ("stages", 128), ("stages", 256))


def divides(box, edge):
    return all(abs(round(L / edge) * edge - L) <= 1e-9 * L for L in box)


def make_batch(boxes, counts, pos, vel, precision, K, edge, lx=0.0, **kw):
    p = D.make_params((1, 1, 1), precision=precision, recompute_every=K, l=edge, lx=lx, **kw)
    b = D.Batch(p, boxes, counts)
    real = b.real
    st = D.BatchState(b, D.to_real4(torch.from_numpy(pos), None, real), D.to_real4(torch.from_numpy(vel), None, real))
    return b, st


def apply_plan(b, plan, size):
    """Select the launch plan and its work size on batch b."""
    D.dcm_batch_set_persistent(b, plan == "persistent")
    if plan == "persistent":
        D.dcm_batch_set_tile(b, size)
    else:
        D.dcm_batch_set_force_block(b, size)


def tune(boxes, counts, pos, vel, precision=D.DCM_PREC_MIXED, K=10, dt=0.005, steps=3, plans=PLANS, **kw):
    """Returns (best (edge, lx, plan, size), {(edge, lx, plan, size): ms per step})."""
    results = {}
    stream = torch.cuda.current_stream()
    for edge, lx in EDGES:
        if not all(divides(b, edge) and divides(b, lx) for b in boxes):
            continue
        b, st = make_batch(boxes, counts, pos, vel, precision, K, edge, lx, **kw)
        D.dcm_batch_step_init(b, st)
        for plan, size in plans:
            apply_plan(b, plan, size)
            D.dcm_batch_step(b, st, dt, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            D.dcm_batch_step(b, st, dt, steps)
            e1.record(stream)
            e1.synchronize()
            results[(edge, lx, plan, size)] = e0.elapsed_time(e1) / steps
        b.close()
    best = min(results, key=results.get)
    return best, results
