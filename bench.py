#!/usr/bin/env python
"""DCM timestep throughput on GB300: particle-steps/s on the 15.5M-particle slab.

One benchmark "step" is one full recomputation period of the dynamic cutoff
method: K = 10 velocity-Verlet timesteps, each with binning, forces and both
half kicks, plus interface detection, fast-sweeping distances and cutoff
assignment once.  So every stage of the hot path runs in every step, and the
reported throughput counts N x 10 particle-timesteps per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  For N > 1 (torchrun) every rank steps its own
independent replica (seed = rank): weak scaling, no data-path collective.
The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on a column of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DCM step particle-steps/s at N=16M"
UNIT = "particle-steps/s"
K_RECOMPUTE = 10
DT = 0.005
REST_BYTES = 197            # HBM bytes per particle and timestep of every stage but the forces:
                            # binning + permutation 96, cell counts/scan 13, velocity Verlet 80,
                            # interface/distances/cutoffs 8 (amortised over the cadence)
LIST_SKIN = 0.5             # Verlet-list skin of the lists form (the fastest measured on the 16M slab)
FLOP_PER_PAIR = 18          # FP32-pipe instructions of the pair arithmetic per accepted pair
FLOP_PER_PAIR_FORCES = 15   # ... without the energy (2) and virial (1) terms: the timesteps of a
                            # dcm_step call before its last, whose energy and virial nothing reads
FP32_LANES_PER_SM = 128
ACC_DESCR = {"fp32": "plain FP32 running sums",
             "plane_kahan": "FP32 per z-plane of the stencil, Kahan-compensated across planes",
             "plane_fp64": "FP32 per z-plane of the stencil, FP64 across planes",
             "row_kahan": "FP32 per row segment, Kahan-compensated across segments",
             "row_fp64": "FP32 per row segment, FP64 across segments",
             "pair_kahan": "every pair term Kahan-compensated in FP32",
             "pair_fp64": "every pair term added in FP64"}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="slab_16m")
    ap.add_argument("--cell-edge", type=float, default=1.5, help="force-cell edge l (density grid h stays 1.5)")
    ap.add_argument("--cell-edge-x", type=float, default=0.5,
                    help="force-cell edge along x, the row direction (0: the cell edge); 0.5 measured fastest "
                         "with the 1.5 cell edge")
    ap.add_argument("--skin", type=float, default=0.0, help="Verlet-list skin (0: forces from cell lists every step)")
    ap.add_argument("--force-kernel", type=int, default=0, help="cell-list force kernel (DCM_FORCE_*; 0: auto)")
    ap.add_argument("--accumulation", type=int, default=0,
                    help="per-particle accumulation of the mixed form (DCM_ACC_*; 0: auto)")
    ap.add_argument("--skip-acc-forms", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-lists", action="store_true")
    ap.add_argument("--skip-adjoint", action="store_true")
    ap.add_argument("--skip-interface", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=500)
    return ap.parse_args(argv)


# ------------------------------------------------------------------ ranks
def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, local, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
        return dist
    return None


def rank_spec(workload: str, rank: int):
    """Each rank steps its own replica of the workload: the same recipe and
    sizes, seeded with the rank (independent systems, no exchange)."""
    from paper_1701_05242_gb300 import synth
    spec = synth.named(workload)
    spec.seed = rank
    return spec


def aggregate(dist, units: float, seconds: float):
    """Whole-job throughput: units summed over ranks, time = max over ranks."""
    if dist is None:
        return units, seconds
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- profiles
FORCE_SOURCES = ("forces_core.cuh", "forces.cu")


def force_source_sha():
    """SHA-256 of the cell-list force kernel's sources (core, then kernels)."""
    h = hashlib.sha256()
    for name in FORCE_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1701_05242_gb300", "csrc", name), "rb").read())
    return h.hexdigest()


def recorded_traffic(workload, cells, acc_name):
    """DRAM bytes per force launch from the committed ncu record
    (profiles/forces_<workload>.json, written beside its Markdown summary), if
    it was taken on the current force kernel sources, the same cell edges
    (l, lx) and the same accumulation form (else None)."""
    path = os.path.join(ROOT, "profiles", f"forces_{workload}.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    if rec.get("forces_src_sha256") != force_source_sha():
        return None
    if tuple(float(c) for c in rec.get("cell_edges", ())) != tuple(cells) or rec.get("accumulation") != acc_name:
        return None
    return float(rec["traffic_bytes_per_launch"])


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# --------------------------------------------------------- CPU baseline
def cpu_sample_spec(workload: str, width: float = 30.0):
    """The same slab recipe (densities, z-profile, surface-wave amplitude,
    seed) on a width x width cross-section: a bounded sample the oracle
    steps in seconds."""
    from paper_1701_05242_gb300 import synth
    spec = synth.named(workload)
    spec.box = (float(width), float(width), float(spec.box[2]))
    spec.name = f"{workload}_cross_section_{width:g}"
    return spec


def oracle_rate(workload, width, nsteps, warmup, nthreads):
    """Particle-steps/s of the FP64 oracle on the cross-section sample, with
    cutoffs recomputed every K_RECOMPUTE steps as in the GPU run."""
    import oracle as O
    from paper_1701_05242_gb300 import synth
    spec = cpu_sample_spec(workload, width)
    slab = synth.make_slab(spec)
    p = O.Params(box=slab.box, recompute_every=K_RECOMPUTE)
    st = O.init_state(slab.pos, slab.vel, p, nthreads=nthreads)
    for _ in range(warmup):
        st = O.step(st, DT, p, nthreads=nthreads)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        st = O.step(st, DT, p, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return slab.n * nsteps / dt, slab.n, dt, slab.box


def oracle_full(slab, nthreads, nsteps=1, warmup=0):
    """The FP64 oracle on the whole workload (the GPU run's configuration):
    nsteps timed timesteps after warmup untimed ones, plus one timed cutoff
    recomputation (interface, distances, cutoffs) charged at 1/K per step, as
    the GPU run recomputes every K steps.  Returns (particle-steps/s, seconds
    per step, seconds per recomputation)."""
    import oracle as O
    p = O.Params(box=slab.box, recompute_every=10 ** 9)   # the timed steps reuse the cutoffs
    st = O.init_state(slab.pos, slab.vel, p, nthreads=nthreads)
    for _ in range(warmup):
        st = O.step(st, DT, p, nthreads=nthreads)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        st = O.step(st, DT, p, nthreads=nthreads)
    t_step = (time.perf_counter() - t0) / max(nsteps, 1)
    t0 = time.perf_counter()
    O.assign_cutoffs(st.pos, p)
    t_rec = time.perf_counter() - t0
    per = t_step + t_rec / K_RECOMPUTE
    return slab.n / per, per, t_rec


# ------------------------------------------------------------------ main
def gpu_config(args, slab, world=1):
    """The workload description both arms print (the same dict)."""
    return {"workload": args.workload, "particles_per_gpu": slab.n, "box": list(slab.box),
            "rc_min": 3.0, "rc_max": 6.0, "h": 1.5, "l": args.cell_edge,
            "lx": args.cell_edge_x if args.cell_edge_x > 0 else args.cell_edge, "skin": args.skin, "dt": DT,
            "recompute_every": K_RECOMPUTE, "thermo_every": K_RECOMPUTE,
            "l2": f"inputs larger than L2 (positions {16 * slab.n / 1e6:.0f} MB)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The FP64 oracle on the host cores, on the whole workload: each bench
    step is one oracle timestep (particle-steps/s as in the GPU arm), plus a
    cutoff recomputation charged at 1/K_RECOMPUTE per timestep (the same
    cadence as the GPU run)."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    from paper_1701_05242_gb300 import synth
    nthreads = os.cpu_count() or 1
    slab = synth.make_slab(rank_spec(args.workload, 0))
    # each bench step: one timed oracle timestep (the warm-up steps untimed)
    rate, per, t_rec = oracle_full(slab, nthreads, nsteps=args.steps, warmup=args.warmup)
    sample = (f"the whole {args.workload} workload ({slab.n} particles): {args.steps} oracle timesteps after "
              f"{args.warmup} untimed ones, plus one cutoff recomputation ({t_rec:.2f} s) charged at 1/{K_RECOMPUTE} "
              f"per timestep; forces threaded with dynamic(20), other stages single-threaded")
    cfg = gpu_config(args, slab)
    out = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
           "timesteps_per_step": 1, "precision": "fp64 (oracle)",
           "warmup": args.warmup, "ms_per_step": 1000.0 * per, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": rate, "unit": UNIT, "cores": nthreads, "kind": "oracle", "sample": sample},
           "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_batch(args, D, dev):
    """64 independent replicas (N log-uniform in [2K, 200K]) stepped together:
    autotuned cell edges and launch plan (persistent, two cooperative launches
    per timestep with a (replica, tile) force queue, or one launch per stage),
    one CUDA graph per recomputation period, args.batch_steps timesteps timed.
    Beside it, on the same replicas: the plain FP64 form (FP64 arrays and
    arithmetic, one launch per stage, no graph)."""
    import numpy as np
    import torch
    from paper_1701_05242_gb300 import autotune, synth
    specs = synth.batch_specs(64)
    slabs = [synth.make_slab(s) for s in specs]
    boxes = [s.box for s in slabs]
    counts = [s.n for s in slabs]
    pos = np.concatenate([s.pos for s in slabs])
    vel = np.concatenate([s.vel for s in slabs])
    best, table = autotune.tune(boxes, counts, pos, vel, K=K_RECOMPUTE, dt=DT)
    b, st = autotune.make_batch(boxes, counts, pos, vel, D.DCM_PREC_MIXED, K_RECOMPUTE, best[0], best[1])
    autotune.apply_plan(b, best[2], best[3])
    D.dcm_batch_step_init(b, st)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    D.dcm_batch_capture(b, st, DT, stream)
    per = D.dcm_batch_graph_steps(b)
    ngraphs = max(1, args.batch_steps // per)
    D.dcm_batch_replay(b, st, 1, stream)
    stream.synchronize()
    D.dcm_batch_launch_count(b, reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    D.dcm_batch_replay(b, st, ngraphs, stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    steps = ngraphs * per
    launches = D.dcm_batch_launch_count(b)
    status = D.dcm_batch_status(b, stream)
    pairs = float(st.thermo.view(-1, 4)[:, 3].sum().item())
    acc = D.ACC_NAMES[D.dcm_batch_accumulation(b)]
    b.close()
    # stage split of both plans (direct stepping with the stage clocks; the
    # timed run above is the graph replay, where no clock runs)
    split = {}
    for plan, size in (("persistent", best[3] if best[2] == "persistent" else 32),
                       ("stages", best[3] if best[2] == "stages" else 256)):
        bp, sp = autotune.make_batch(boxes, counts, pos, vel, D.DCM_PREC_MIXED, K_RECOMPUTE, best[0], best[1])
        autotune.apply_plan(bp, plan, size)
        D.dcm_batch_step_init(bp, sp)
        D.dcm_batch_step(bp, sp, DT, K_RECOMPUTE)
        D.dcm_batch_set_timing(bp, 8192)
        D.dcm_batch_stage_times(bp)
        D.dcm_batch_launch_count(bp, reset=True)
        e0.record()
        D.dcm_batch_step(bp, sp, DT, 2 * K_RECOMPUTE)
        e1.record()
        e1.synchronize()
        st_ms = D.dcm_batch_stage_times(bp)
        split[f"{plan}={size}"] = {"ms_per_timestep": e0.elapsed_time(e1) / (2 * K_RECOMPUTE),
                                   "launches_per_timestep": D.dcm_batch_launch_count(bp) / (2 * K_RECOMPUTE),
                                   "stage_ms_per_timestep": {k: v[0] / (2 * K_RECOMPUTE) for k, v in st_ms.items()}}
        bp.close()
    # the plain FP64 form on the same replicas: per-stage launches, no graph
    b64, s64 = autotune.make_batch(boxes, counts, pos, vel, D.DCM_PREC_FP64, K_RECOMPUTE, 1.5, 0.0)
    D.dcm_batch_set_persistent(b64, False)
    D.dcm_batch_step_init(b64, s64)
    D.dcm_batch_step(b64, s64, DT, 1)
    n64 = K_RECOMPUTE
    torch.cuda.synchronize()
    e0.record()
    D.dcm_batch_step(b64, s64, DT, n64)
    e1.record()
    e1.synchronize()
    ms64 = e0.elapsed_time(e1)
    status64 = D.dcm_batch_status(b64)
    b64.close()
    value = sum(counts) * steps / (ms / 1000.0)
    value64 = sum(counts) * n64 / (ms64 / 1000.0)
    out = {"value": value, "unit": UNIT, "replicas": len(counts),
           "particles": int(sum(counts)), "n_min": int(min(counts)), "n_max": int(max(counts)),
           "timesteps": steps, "ms_per_timestep": ms / steps, "cuda_graph": True,
           "graph_timesteps": per, "launches_per_timestep": launches / steps,
           "plan": best[2], "tile_or_block": best[3], "accumulation": acc, "pairs_per_timestep": pairs,
           "autotuned": {"cell_edge": best[0], "cell_edge_x": best[1], "plan": best[2], "size": best[3],
                         "candidates_ms": {f"l={k[0]},lx={k[1]},{k[2]}={k[3]}": v for k, v in table.items()}},
           "plain_fp64_form": {"value": value64, "unit": UNIT, "timesteps": n64, "ms_per_timestep": ms64 / n64,
                               "plan": "stages", "cuda_graph": False, "device_status": status64},
           "speedup_over_plain_fp64": value / value64,
           "plans_direct_stepping": split,
           "device_status": status}
    return out


def run_interface_forms(args, D, dev, slab, ps):
    """The interface stage's forms on the benchmark's box grid (16.4M density
    boxes of 1.5 at 16M), from the box counts of the sorted positions ps:
    the default 2-means threshold of the smoothed counts, the regularised
    two-phase segmentation with its length term (Section 2.1; nu = 4, 200
    inner and 4 outer iterations), and the default with the bubble filter
    (components under 20 boxes removed); then the whole timestep on the
    curved (cylindrical) interface workload.  CUDA events on the launching
    stream, three repetitions each after one untimed."""
    import torch
    from paper_1701_05242_gb300 import synth
    stream = torch.cuda.current_stream(dev)
    n = ps.shape[0]
    i32 = dict(dtype=torch.int32, device=dev)
    out = {"boxes": None}
    ref_s = None
    for name, kw in (("two_means", {}), ("regularised", dict(segmentation=1, ms_nu=4.0, ms_inner=200, ms_outer=4)),
                     ("bubble_filter", dict(min_component=20))):
        p = D.make_params(slab.box, n_max=n, l=args.cell_edge, lx=args.cell_edge_x, **kw)
        c = D.Context(p)
        bc = torch.empty(c.nbox, **i32)
        s = torch.empty(c.nbox, dtype=torch.uint8, device=dev)
        iface = torch.empty_like(s)
        thr = torch.empty(1, **i32)
        D.dcm_box_counts(c, n, ps, bc)
        D.dcm_detect_interface(c, bc, s, iface, thr)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(3):
            D.dcm_detect_interface(c, bc, s, iface, thr)
        ev1.record(stream)
        ev1.synchronize()
        rec = {"ms": ev0.elapsed_time(ev1) / 3, "interface_boxes": int(iface.sum().item()),
               "device_status": D.dcm_status(c)}
        if ref_s is None:
            ref_s = s.clone()
            out["boxes"] = int(c.nbox)
        else:
            rec["boxes_changed"] = int((s != ref_s).sum().item())
        out[name] = rec
        c.close()
        del bc, s, iface
    torch.cuda.empty_cache()
    cyl = synth.make_slab(synth.named("cylinder_299k"))
    p = D.make_params(cyl.box, n_max=cyl.n, recompute_every=K_RECOMPUTE, l=args.cell_edge, lx=args.cell_edge_x)
    c = D.Context(p)
    stc = D.State(c, D.to_real4(torch.from_numpy(cyl.pos), None, torch.float32, dev),
                  D.to_real4(torch.from_numpy(cyl.vel), None, torch.float32, dev))
    D.dcm_step_init(c, stc)
    D.dcm_step(c, stc, DT, K_RECOMPUTE)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(5):
        D.dcm_step(c, stc, DT, K_RECOMPUTE)
    ev1.record(stream)
    ev1.synchronize()
    msc = ev0.elapsed_time(ev1)
    out["cylinder_299k"] = {"value": cyl.n * 5 * K_RECOMPUTE / (msc / 1000.0), "unit": UNIT, "particles": cyl.n,
                            "timesteps": 5 * K_RECOMPUTE, "device_status": D.dcm_status(c)}
    c.close()
    return out


def run_adjoint(args, D, dev):
    """Differentiation form on the two-type workload (260,522 particles,
    per-type eps and sigma, Lorentz-Berthelot): cutoffs from the method's own
    stages, then the force evaluation and the hand-written adjoint of
    L = sum_i |F_i|^2 + E (cutoffs held fixed), each timed with CUDA events on
    the launching stream, in both precision forms."""
    import torch
    from paper_1701_05242_gb300 import synth
    slab = synth.make_slab(synth.named("slab_256k_2types"))
    n = slab.n
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "slab_256k_2types", "particles": n, "unit": "particle-gradients/s",
           "loss": "sum_i |F_i|^2 + E, cutoffs held fixed"}
    for prec, key in ((D.DCM_PREC_MIXED, "mixed"), (D.DCM_PREC_FP64, "fp64")):
        p = D.make_params(slab.box, n_max=n, precision=prec, ntypes=2, eps=(1.0, 0.8), sigma=(1.0, 1.1),
                          l=args.cell_edge, lx=args.cell_edge_x)
        ctx = D.Context(p)
        real = ctx.real
        pos4 = D.to_real4(torch.from_numpy(slab.pos), torch.from_numpy(slab.types), real, dev)
        i32 = dict(dtype=torch.int32, device=dev)
        cell, start, perm = torch.empty(n, **i32), torch.empty(ctx.ncell + 1, **i32), torch.empty(n, **i32)
        ps = torch.empty_like(pos4)
        D.dcm_bin(ctx, n, pos4, cell, start, perm, ps)
        bc, g = torch.empty(ctx.nbox, **i32), torch.empty(ctx.nbox, **i32)
        s = torch.empty(ctx.nbox, dtype=torch.uint8, device=dev)
        iface = torch.empty_like(s)
        thr = torch.empty(1, **i32)
        D.dcm_box_counts(ctx, n, ps, bc)
        D.dcm_detect_interface(ctx, bc, s, iface, thr, g)
        dist = torch.empty(ctx.nbox, dtype=real, device=dev)
        D.dcm_distance(ctx, s, iface, dist)
        rc = torch.empty(n, dtype=real, device=dev)
        D.dcm_cutoffs(ctx, n, ps, dist, rc)
        F = torch.empty_like(ps)
        tot = torch.zeros(3, dtype=torch.float64, device=dev)
        A = torch.zeros_like(ps)
        G = torch.empty_like(ps)
        dpar = torch.zeros(4, dtype=torch.float64, device=dev)
        reps = 10 if prec == D.DCM_PREC_MIXED else 3
        fwd_ms = bwd_ms = 0.0
        for it in range(3 + reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            D.dcm_forces(ctx, n, ps, rc, start, F, tot)
            ev[1].record(stream)
            A[:, :3] = 2.0 * F[:, :3]  # dL/dF
            ev[2].record(stream)
            D.dcm_forces_backward(ctx, n, ps, rc, start, A, 1.0, G, dpar)
            ev[3].record(stream)
            ev[3].synchronize()
            if it >= 3:
                fwd_ms += ev[0].elapsed_time(ev[1]) / reps
                bwd_ms += ev[2].elapsed_time(ev[3]) / reps
        out[key] = {"forward_ms": fwd_ms, "backward_ms": bwd_ms, "backward_over_forward": bwd_ms / fwd_ms,
                    "value": n / ((fwd_ms + bwd_ms) / 1000.0), "device_status": D.dcm_status(ctx)}
        ctx.close()
    out["value"] = out["mixed"]["value"]
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def run_gb300(args):
    import numpy as np
    import torch

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = dist_init(world, local, "nccl")
    import paper_1701_05242_gb300.dcm as D
    from paper_1701_05242_gb300 import synth

    slab = synth.make_slab(rank_spec(args.workload, rank))
    n = slab.n
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    def new_state(prec, skin=None, newton3=0):
        p = D.make_params(slab.box, n_max=n, precision=prec, recompute_every=K_RECOMPUTE, l=args.cell_edge,
                          lx=args.cell_edge_x, skin=args.skin if skin is None else skin,
                          force_kernel=args.force_kernel, accumulation=args.accumulation, newton3=newton3)
        ctx = D.Context(p)
        real = ctx.real
        st = D.State(ctx, D.to_real4(torch.from_numpy(slab.pos), None, real, dev),
                      D.to_real4(torch.from_numpy(slab.vel), None, real, dev))
        D.dcm_step_init(ctx, st)
        return ctx, st

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- mixed form: the timed path
    ctx, st = new_state(D.DCM_PREC_MIXED)
    for _ in range(args.warmup):
        D.dcm_step(ctx, st, DT, K_RECOMPUTE)
    barrier()
    D.dcm_set_timing(ctx, args.steps * K_RECOMPUTE + 8)
    D.dcm_launch_count(ctx, reset=True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        D.dcm_step(ctx, st, DT, K_RECOMPUTE)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    launches = D.dcm_launch_count(ctx)
    stages = D.dcm_stage_times(ctx)
    thermo = st.thermo.cpu().numpy()
    status = D.dcm_status(ctx)
    barrier()
    units = float(n) * args.steps * K_RECOMPUTE
    tot_units, secs = aggregate(dist, units, ms / 1000.0)
    value = tot_units / secs

    # the same path with energy, virial and thermo on every timestep (one
    # dcm_step call per timestep), for comparison with the headline's
    # thermo once per call of K timesteps
    kt = 2 * K_RECOMPUTE
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(stream)
    for _ in range(kt):
        D.dcm_step(ctx, st, DT, 1)
    t1.record(stream)
    torch.cuda.synchronize()
    ue1, te1 = aggregate(dist, float(n) * kt, t0.elapsed_time(t1) / 1000.0)
    every_ts = {"value": ue1 / te1, "unit": UNIT, "timesteps": kt,
                "note": "one dcm_step call per timestep: energy, virial and thermo every timestep"}

    # roofline of the dominant kernel (forces): FP32-pipe instructions
    f_ms, f_cnt = stages["forces"]
    pairs = float(thermo[3])
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = measured_peaks()
    fmax = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tinstr = sms * FP32_LANES_PER_SM * fmax * 1e6 / 1e12
    f_avg_s = (f_ms / max(f_cnt, 1)) / 1000.0
    # one launch per dcm_step call (its last timestep) sums energy and virial
    n_ew = min(args.steps, f_cnt)
    instr_pp = (FLOP_PER_PAIR * n_ew + FLOP_PER_PAIR_FORCES * (f_cnt - n_ew)) / max(f_cnt, 1)
    achieved = pairs * instr_pp / f_avg_s / 1e12 if f_avg_s > 0 else None
    fkern = "k_forces_list" if args.skin > 0 else D.FORCE_KERNEL_NAMES[D.dcm_force_kernel(ctx)]
    acc_name = D.ACC_NAMES[D.dcm_accumulation(ctx)]
    cells = (args.cell_edge, args.cell_edge_x if args.cell_edge_x > 0 else args.cell_edge)
    roof = {"bound": "alu", "kernel": fkern, "achieved": achieved, "peak": peak_tinstr,
            "unit": "T FP32-instr/s", "frac": (achieved / peak_tinstr) if achieved else None,
            "traffic": recorded_traffic(args.workload, cells, acc_name),
            "avg_launch_ms": f_ms / max(f_cnt, 1),
            "pairs_per_launch": pairs, "instr_per_pair": instr_pp,
            "instr_basis": f"{FLOP_PER_PAIR} per pair in the {n_ew} launches that sum energy and virial, "
                           f"{FLOP_PER_PAIR_FORCES} in the other {f_cnt - n_ew}",
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x {fmax:g} MHz (max clock)"}
    stage_ms = {k: v[0] / max(args.steps, 1) for k, v in stages.items()}
    # step roofline: the force kernel at the FP32-pipe peak plus every other
    # stage at the measured HBM bandwidth (REST_BYTES per particle per timestep)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    f_ideal = pairs * instr_pp / (peak_tinstr * 1e12) * 1e3
    r_ideal = n * REST_BYTES / (hbm * 1e9) * 1e3
    t_meas = ms / max(args.steps * K_RECOMPUTE, 1)
    step_roof = {"force_ideal_ms": f_ideal, "rest_ideal_ms": r_ideal, "ideal_ms_per_timestep": f_ideal + r_ideal,
                 "measured_ms_per_timestep": t_meas, "frac": (f_ideal + r_ideal) / t_meas if t_meas > 0 else None,
                 "basis": f"pairs x {instr_pp:.2f} FP32-pipe instr at the peak above + {REST_BYTES} B/particle "
                          f"at {hbm:g} GB/s (measured copy bandwidth)"}

    # ---------------- the force launch in every per-particle accumulation form,
    # on the final sorted state of the timed run (CUDA events, same stream)
    acc_forms = None
    if not args.skip_acc_forms and args.skin == 0.0:
        acc_forms = {}
        ps, _, rcs, _ = st.current()
        starts = torch.empty(ctx.ncell + 1, dtype=torch.int32, device=dev)
        cellb = torch.empty(n, dtype=torch.int32, device=dev)
        permb = torch.empty(n, dtype=torch.int32, device=dev)
        pss = torch.empty_like(ps)
        D.dcm_bin(ctx, n, ps, cellb, starts, permb, pss)
        rcss = rcs[permb.long()]
        Fb = torch.empty_like(pss)
        totb = torch.zeros(3, dtype=torch.float64, device=dev)
        for acc in (D.DCM_ACC_FP32, D.DCM_ACC_PLANE_KAHAN, D.DCM_ACC_PLANE_FP64, D.DCM_ACC_ROW_KAHAN,
                    D.DCM_ACC_ROW_FP64, D.DCM_ACC_PAIR_KAHAN, D.DCM_ACC_PAIR_FP64):
            pa = D.make_params(slab.box, n_max=n, recompute_every=K_RECOMPUTE, l=args.cell_edge,
                               lx=args.cell_edge_x, force_kernel=args.force_kernel, accumulation=acc)
            ca = D.Context(pa)
            D.dcm_forces(ca, n, pss, rcss, starts, Fb, totb)
            reps = 5
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(reps):
                D.dcm_forces(ca, n, pss, rcss, starts, Fb, totb)
            a1.record(stream)
            a1.synchronize()
            ams = a0.elapsed_time(a1) / reps
            pa_pairs = float(totb[2].item())
            acc_forms[D.ACC_NAMES[acc]] = {"ms_per_launch": ams, "E": float(totb[0].item()),
                                           "W": float(totb[1].item()), "pairs": pa_pairs,
                                           "frac": pa_pairs * FLOP_PER_PAIR / (ams / 1000.0) / 1e12 / peak_tinstr}
            ca.close()
        del pss, Fb, rcss, starts, cellb, permb

    # ---------------- plain FP64 form on the same GPU (per-step launches)
    fp64 = None
    if not args.skip_fp64:
        del st
        ctx.close()
        torch.cuda.empty_cache()
        c64, s64 = new_state(D.DCM_PREC_FP64)
        D.dcm_step(c64, s64, DT, K_RECOMPUTE)
        k64 = max(1, min(2, args.steps))
        barrier()
        e0.record(stream)
        for _ in range(k64):
            D.dcm_step(c64, s64, DT, K_RECOMPUTE)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        u64, t64 = aggregate(dist, float(n) * k64 * K_RECOMPUTE, ms64 / 1000.0)
        fp64 = {"value": u64 / t64, "unit": UNIT, "steps": k64, "ms_per_step": ms64 / k64,
                "speedup_mixed_over_fp64": value / (u64 / t64), "device_status": D.dcm_status(c64)}
        del s64
        c64.close()
        torch.cuda.empty_cache()
        ctx, st = new_state(D.DCM_PREC_MIXED)

    # ---------------- end to end through the public API with host buffers
    e2e = None
    if not args.skip_e2e:
        # A stream of independent jobs, each: the state in from pinned host
        # memory, dcm_step_init + 10 timesteps, state and thermo back out.
        # Two device states take turns, so job j+1's copy in and job j-1's
        # copy out run on a copy stream while job j computes.
        pos_h = D.to_real4(torch.from_numpy(slab.pos), None, torch.float32, "cpu").pin_memory()
        vel_h = D.to_real4(torch.from_numpy(slab.vel), None, torch.float32, "cpu").pin_memory()
        outs = [(torch.empty_like(pos_h).pin_memory(), torch.empty_like(vel_h).pin_memory(),
                 torch.empty(4, dtype=torch.float64).pin_memory()) for _ in range(2)]
        sts = [st, D.State(ctx, D.to_real4(torch.from_numpy(slab.pos), None, torch.float32, dev),
                           D.to_real4(torch.from_numpy(slab.vel), None, torch.float32, dev))]
        cs = torch.cuda.Stream(dev)
        h2d_ev = [torch.cuda.Event() for _ in range(2)]
        comp_ev = [torch.cuda.Event() for _ in range(2)]
        ke = max(2, min(6, args.steps))

        def h2d(j):
            s = sts[j % 2]
            with torch.cuda.stream(cs):
                k = s.c.cur
                s.pos[k].copy_(pos_h, non_blocking=True)
                s.vel[k].copy_(vel_h, non_blocking=True)
                h2d_ev[j % 2].record(cs)

        def compute(j):
            s = sts[j % 2]
            stream.wait_event(h2d_ev[j % 2])
            D.dcm_step_init(ctx, s, stream)
            D.dcm_step(ctx, s, DT, K_RECOMPUTE, stream)
            comp_ev[j % 2].record(stream)

        def d2h(j):
            s, (po, vo, to) = sts[j % 2], outs[j % 2]
            cs.wait_event(comp_ev[j % 2])
            with torch.cuda.stream(cs):
                k = s.c.cur
                po.copy_(s.pos[k], non_blocking=True)
                vo.copy_(s.vel[k], non_blocking=True)
                to.copy_(s.thermo, non_blocking=True)

        def jobs(count, t0=None, t1=None):
            if t0 is not None:
                t0.record(cs)
            h2d(0)
            for j in range(count):
                if j + 1 < count:
                    h2d(j + 1)
                compute(j)
                d2h(j)
            if t1 is not None:
                t1.record(cs)

        jobs(2)
        torch.cuda.synchronize()
        barrier()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        jobs(ke, t0, t1)
        torch.cuda.synchronize()
        mse = t0.elapsed_time(t1)
        ue, te = aggregate(dist, float(n) * ke * K_RECOMPUTE, mse / 1000.0)
        e2e = {"value": ue / te, "unit": UNIT, "h2d_bytes_per_step": 2 * n * 16,
               "d2h_bytes_per_step": 2 * n * 16 + 32, "steps": ke,
               "note": "per step a job: pinned host state in, dcm_step_init + 10 timesteps, state and thermo out; "
                       "two device states alternate so that the copies of the neighbouring jobs run on a copy "
                       "stream during a job's compute"}
        del sts

    # ---------------- Verlet-list forms (Alg. 2.2/2.3 with skin) on the same system:
    # full i-centric lists, and half lists with Newton's third law
    lists = lists_n3 = None
    if not args.skip_lists and args.skin == 0.0:
        del st
        ctx.close()
        torch.cuda.empty_cache()
        for newton3 in (0, 1):
            cl, sl = new_state(D.DCM_PREC_MIXED, skin=LIST_SKIN, newton3=newton3)
            for _ in range(args.warmup):
                D.dcm_step(cl, sl, DT, K_RECOMPUTE)
            kl = max(1, min(10, args.steps))
            barrier()
            D.dcm_set_timing(cl, kl * K_RECOMPUTE * 2 + 8)
            e0.record(stream)
            for _ in range(kl):
                D.dcm_step(cl, sl, DT, K_RECOMPUTE)
            e1.record(stream)
            torch.cuda.synchronize()
            msl = e0.elapsed_time(e1)
            lst = D.dcm_stage_times(cl)
            pl = float(sl.thermo[3].item())
            ul, tl = aggregate(dist, float(n) * kl * K_RECOMPUTE, msl / 1000.0)
            lf_ms, lf_cnt = lst["forces"]
            lf_avg = lf_ms / max(lf_cnt, 1)
            # the list kernels sum energy and virial on every timestep
            l_ew = lf_cnt
            l_ipp = (FLOP_PER_PAIR * l_ew + FLOP_PER_PAIR_FORCES * (lf_cnt - l_ew)) / max(lf_cnt, 1)
            rec = {"value": ul / tl, "unit": UNIT, "steps": kl, "ms_per_step": msl / kl, "skin": LIST_SKIN,
                   "force_kernel": "k_forces_list_n3_x2" if newton3 else "k_forces_list_x2",
                   "force_avg_launch_ms": lf_avg,
                   "force_frac_fp32": pl * l_ipp / (lf_avg / 1000.0) / 1e12 / peak_tinstr if lf_avg > 0 else None,
                   "instr_per_pair": l_ipp,
                   "list_builds": int(lst["lists"][1]), "build_avg_ms": lst["lists"][0] / max(lst["lists"][1], 1),
                   "stage_ms_per_step": {k: v[0] / kl for k, v in lst.items()}, "pairs_last": pl,
                   "device_status": D.dcm_status(cl),
                   "note": ("half lists kept by the larger-cutoff particle, each pair evaluated once and scattered "
                            "(atomics) to the other particle where its cutoff reaches" if newton3 else
                            "neighbour lists of radius rc_i + skin") +
                           ", rebuilt (with rebinning) when a particle moved more than skin/2 or the cutoffs were "
                           "recomputed"}
            if newton3:
                lists_n3 = rec
            else:
                lists = rec
            del sl
            cl.close()
            torch.cuda.empty_cache()
        ctx, st = new_state(D.DCM_PREC_MIXED)

    # ---------------- interface forms (f1, f2) on the same box grid
    interface = None
    if not args.skip_interface and rank == 0:
        ps_i, _, _, _ = st.current()
        interface = run_interface_forms(args, D, dev, slab, ps_i)
        del ps_i
        torch.cuda.empty_cache()

    # ---------------- batched form: 64 replicas, autotuned, graph-captured
    batch = adjoint = None
    if not args.skip_batch or not args.skip_adjoint:
        del st
        ctx.close()
        torch.cuda.empty_cache()
    if not args.skip_batch:
        batch = run_batch(args, D, dev)
    if not args.skip_adjoint and rank == 0:
        adjoint = run_adjoint(args, D, dev)

    # ---------------- CPU oracle on the host cores (rank 0, N = 1): the whole
    # workload on all cores; one core on a cross-section (context)
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        nthreads = os.cpu_count() or 1
        rate, per, t_rec = oracle_full(slab, nthreads)
        rate1, n_s, _, box = oracle_rate(args.workload, 30.0, 3, 1, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": nthreads, "kind": "oracle",
               "sample": f"the whole {args.workload} workload ({n} particles): one oracle timestep plus one cutoff "
                         f"recomputation ({t_rec:.2f} s) charged at 1/{K_RECOMPUTE} (cell-list forces threaded with "
                         f"dynamic(20), other stages single-threaded)",
               "single_thread_value": rate1,
               "single_thread_sample": f"{n_s} particles ({box[0]:g}x{box[1]:g}x{box[2]:g} cross-section of the "
                                       f"same recipe), 3 timesteps on one core"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": secs * 1000.0 / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": gpu_config(args, slab, world), "timesteps_per_step": K_RECOMPUTE,
               "precision": f"fp32 pair math, per-particle sums {acc_name} "
                            f"({ACC_DESCR.get(acc_name, acc_name)}), fp64 totals",
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
               "stage_ms_per_step": stage_ms, "step_roofline": step_roof, "thermo_every_timestep": every_ts,
               "accumulation_forms": acc_forms, "fp64_form": fp64, "lists_form": lists, "lists_newton3_form": lists_n3, "batched_form": batch,
               "adjoint_form": adjoint, "interface_forms": interface, "device_status": status,
               "thermo_last": {"E": float(thermo[0]), "W": float(thermo[1]), "KE": float(thermo[2]),
                               "pairs": pairs}}
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
