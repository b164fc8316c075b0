"""Autotuner for the batched form: picks the force-cell edges (l, and lx
along the rows) and the force kernel's block size by timing a few steps of
every candidate on the actual replicas (CUDA events on the stepping stream).

Candidates: (l, lx) in {(1.5, 1.5), (1.5, 0.75), (1.5, 0.5), (1.0, 1.0),
(0.75, 0.75)} where both divide every replica box (h = 1.5 stays the
density-grid edge), block sizes {64, 128, 256}.
"""
from __future__ import annotations

import numpy as np
import torch

from . import dcm as D

EDGES = ((1.5, 1.5), (1.5, 0.75), (1.5, 0.5), (1.0, 1.0), (0.75, 0.75))
BLOCKS = (64, 128, 256)


def divides(box, edge):
    return all(abs(round(L / edge) * edge - L) <= 1e-9 * L for L in box)


def make_batch(boxes, counts, pos, vel, precision, K, edge, lx=0.0, **kw):
    p = D.make_params((1, 1, 1), precision=precision, recompute_every=K, l=edge, lx=lx, **kw)
    b = D.Batch(p, boxes, counts)
    real = b.real
    st = D.BatchState(b, D.to_real4(torch.from_numpy(pos), None, real), D.to_real4(torch.from_numpy(vel), None, real))
    return b, st


def tune(boxes, counts, pos, vel, precision=D.DCM_PREC_MIXED, K=10, dt=0.005, steps=3, **kw):
    """Returns (best (edge, lx, block), {(edge, lx, block): ms per step})."""
    results = {}
    stream = torch.cuda.current_stream()
    for edge, lx in EDGES:
        if not all(divides(b, edge) and divides(b, lx) for b in boxes):
            continue
        b, st = make_batch(boxes, counts, pos, vel, precision, K, edge, lx, **kw)
        D.dcm_batch_step_init(b, st)
        for bs in BLOCKS:
            D.dcm_batch_set_force_block(b, bs)
            D.dcm_batch_step(b, st, dt, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            D.dcm_batch_step(b, st, dt, steps)
            e1.record(stream)
            e1.synchronize()
            results[(edge, lx, bs)] = e0.elapsed_time(e1) / steps
        b.close()
    best = min(results, key=results.get)
    return best, results
