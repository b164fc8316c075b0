"""Python binding of libdcm (include/dcm.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
torch tensors as raw device pointers plus the current CUDA stream; all work
happens in the library's CUDA kernels.  There is no CPU fallback: if the
library cannot be built or loaded, importing this module raises.

Array conventions (see include/dcm.h):
  precision MIXED: real4 = float32 tensor of shape (n, 4), real = float32
  precision FP64:  real4 = float64 tensor of shape (n, 4), real = float64
  positions (x, y, z, type), forces (fx, fy, fz, e_i).
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

DCM_OK = 0
DCM_ERR_INVALID_ARG = 1
DCM_ERR_BOX = 2
DCM_ERR_CUDA = 3
DCM_ERR_NOT_CONVERGED = 4
DCM_ERR_CAPACITY = 5
DCM_ERR_NOMEM = 6
DCM_ERR_TIMEOUT = 7
DCM_PREC_FP64 = 0
DCM_PREC_MIXED = 1
DCM_FORCE_AUTO = 0
DCM_FORCE_THREAD = 1
DCM_FORCE_PACKED = 3
DCM_ACC_AUTO = 0
DCM_ACC_FP32 = 1
DCM_ACC_ROW_FP64 = 2
DCM_ACC_ROW_KAHAN = 3
DCM_ACC_PAIR_KAHAN = 4
DCM_ACC_PAIR_FP64 = 5
DCM_ACC_PLANE_FP64 = 6
DCM_ACC_PLANE_KAHAN = 7
ACC_NAMES = {DCM_ACC_FP32: "fp32", DCM_ACC_ROW_FP64: "row_fp64", DCM_ACC_ROW_KAHAN: "row_kahan",
             DCM_ACC_PAIR_KAHAN: "pair_kahan", DCM_ACC_PAIR_FP64: "pair_fp64", DCM_ACC_PLANE_FP64: "plane_fp64",
             DCM_ACC_PLANE_KAHAN: "plane_kahan"}

_ERRNAMES = {1: "INVALID_ARG", 2: "BOX", 3: "CUDA", 4: "NOT_CONVERGED", 5: "CAPACITY", 6: "NOMEM", 7: "TIMEOUT"}


class DcmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"DCM_ERR_{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class dcm_params(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("h", ctypes.c_double), ("l", ctypes.c_double),
                ("rc_min", ctypes.c_double), ("rc_max", ctypes.c_double), ("ramp", ctypes.c_double),
                ("r_grid", ctypes.c_double), ("smooth_w", ctypes.c_int32), ("threshold", ctypes.c_int32),
                ("iter_max", ctypes.c_int32), ("ntypes", ctypes.c_int32), ("eps", ctypes.c_double * 4),
                ("sigma", ctypes.c_double * 4), ("shift_energy", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("recompute_every", ctypes.c_int32), ("force_kernel", ctypes.c_int32), ("n_max", ctypes.c_int64),
                ("skin", ctypes.c_double), ("min_component", ctypes.c_int32), ("accumulation", ctypes.c_int32),
                ("lx", ctypes.c_double), ("newton3", ctypes.c_int32),
                ("segmentation", ctypes.c_int32), ("ms_inner", ctypes.c_int32), ("ms_outer", ctypes.c_int32),
                ("reserved4", ctypes.c_int32), ("ms_nu", ctypes.c_double)]


class dcm_state(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p * 2), ("vel", ctypes.c_void_p * 2), ("rc", ctypes.c_void_p * 2),
                ("id", ctypes.c_void_p * 2), ("force", ctypes.c_void_p), ("thermo", ctypes.c_void_p),
                ("cur", ctypes.c_int32), ("reserved", ctypes.c_int32), ("t", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_SIGS = {
    "dcm_params_default": (_i32, [ctypes.POINTER(dcm_params)]),
    "dcm_validate_params": (_i32, [ctypes.POINTER(dcm_params), ctypes.c_char_p, _i32]),
    "dcm_grid_dims": (_i32, [ctypes.POINTER(dcm_params), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "dcm_scratch_bytes": (_i32, [ctypes.POINTER(dcm_params), ctypes.POINTER(_i64)]),
    "dcm_version": (ctypes.c_char_p, []),
    "dcm_create": (_i32, [ctypes.POINTER(dcm_params), ctypes.POINTER(_vp)]),
    "dcm_destroy": (None, [_vp]),
    "dcm_last_error": (ctypes.c_char_p, [_vp]),
    "dcm_status": (_i32, [_vp, _vp]),
    "dcm_bin": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dcm_box_counts": (_i32, [_vp, _i64, _vp, _vp, _vp]),
    "dcm_detect_interface": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dcm_remove_small_components": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "dcm_distance": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "dcm_cutoffs": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "dcm_forces": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dcm_step_init": (_i32, [_vp, ctypes.POINTER(dcm_state), _i64, _vp]),
    "dcm_step": (_i32, [_vp, ctypes.POINTER(dcm_state), _i64, ctypes.c_double, _i32, _vp]),
    "dcm_distance_noalloc": (_i32, [ctypes.POINTER(dcm_params), _vp, _vp, _vp, _vp, _vp]),
    "dcm_batch_create": (_i32, [ctypes.POINTER(dcm_params), _i32, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(_i64), ctypes.POINTER(_vp)]),
    "dcm_batch_destroy": (None, [_vp]),
    "dcm_batch_last_error": (ctypes.c_char_p, [_vp]),
    "dcm_batch_offsets": (_i32, [_vp, ctypes.POINTER(_i64)]),
    "dcm_batch_set_force_block": (_i32, [_vp, _i32]),
    "dcm_batch_step_init": (_i32, [_vp, ctypes.POINTER(dcm_state), _vp]),
    "dcm_batch_step": (_i32, [_vp, ctypes.POINTER(dcm_state), ctypes.c_double, _i32, _vp]),
    "dcm_batch_capture": (_i32, [_vp, ctypes.POINTER(dcm_state), ctypes.c_double, _vp]),
    "dcm_batch_replay": (_i32, [_vp, ctypes.POINTER(dcm_state), _i32, _vp]),
    "dcm_batch_graph_steps": (_i32, [_vp]),
    "dcm_batch_set_persistent": (_i32, [_vp, _i32]),
    "dcm_batch_set_wait_budget": (_i32, [_vp, _i64]),
    "dcm_batch_set_tile": (_i32, [_vp, _i32]),
    "dcm_batch_accumulation": (_i32, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "dcm_batch_barrier_selftest": (_i32, [_vp, _i32, _i64, _vp]),
    "dcm_scan_wait_selftest": (_i32, [_vp, _vp]),
    "dcm_batch_status": (_i32, [_vp, _vp]),
    "dcm_batch_set_timing": (_i32, [_vp, _i32]),
    "dcm_batch_stage_times": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)]),
    "dcm_batch_launch_count": (_i32, [_vp, ctypes.POINTER(_i64), _i32]),
    "dcm_set_lj": (_i32, [_vp, _i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "dcm_forces_backward": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
    "dcm_set_timing": (_i32, [_vp, _i32]),
    "dcm_stage_times": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)]),
    "dcm_launch_count": (_i32, [_vp, ctypes.POINTER(_i64), _i32]),
    "dcm_force_kernel": (_i32, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "dcm_accumulation": (_i32, [_vp, ctypes.POINTER(ctypes.c_int32)]),
}

STAGES = ("kick_drift", "bin", "detect", "distance", "cutoffs", "forces", "kick", "lists")


def _load_library():
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib, path


lib, LIB_PATH = _load_library()


def exported_names():
    return list(_SIGS)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("device tensors are required (the library has no CPU path)")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """Owns one dcm_ctx (library scratch) for a parameter set."""

    def __init__(self, params: dcm_params):
        self.params = params
        h = ctypes.c_void_p()
        rc = lib.dcm_create(ctypes.byref(params), ctypes.byref(h))
        if rc != DCM_OK:
            msg = ctypes.create_string_buffer(512)
            lib.dcm_validate_params(ctypes.byref(params), msg, 512)
            raise DcmError(rc, msg.value.decode() or "dcm_create failed")
        self.handle = h
        cells = (_i64 * 3)()
        boxes = (_i64 * 3)()
        lib.dcm_grid_dims(ctypes.byref(params), cells, boxes)
        self.cells = tuple(cells)
        self.boxes = tuple(boxes)
        self.ncell = cells[0] * cells[1] * cells[2]
        self.nbox = boxes[0] * boxes[1] * boxes[2]
        self.real = torch.float32 if params.precision == DCM_PREC_MIXED else torch.float64

    def check(self, rc):
        if rc != DCM_OK:
            raise DcmError(rc, lib.dcm_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            lib.dcm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(box, **kw) -> dcm_params:
    p = dcm_params()
    lib.dcm_params_default(ctypes.byref(p))
    for d in range(3):
        p.box[d] = float(box[d])
    for k, v in kw.items():
        if k in ("eps", "sigma"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = float(x)
        else:
            setattr(p, k, v)
    return p


def dcm_validate_params(p: dcm_params):
    msg = ctypes.create_string_buffer(512)
    rc = lib.dcm_validate_params(ctypes.byref(p), msg, 512)
    return rc, msg.value.decode()


def dcm_status(ctx: Context, stream=None):
    return lib.dcm_status(ctx.handle, _stream(stream))


def dcm_bin(ctx: Context, n, pos, cell, cell_start, perm, pos_sorted=None, stream=None):
    ctx.check(lib.dcm_bin(ctx.handle, n, _ptr(pos), _ptr(cell), _ptr(cell_start), _ptr(perm), _ptr(pos_sorted),
                          _stream(stream)))


def dcm_box_counts(ctx: Context, n, pos, box_count, stream=None):
    ctx.check(lib.dcm_box_counts(ctx.handle, n, _ptr(pos), _ptr(box_count), _stream(stream)))


def dcm_detect_interface(ctx: Context, box_count, s, iface, threshold, g=None, stream=None):
    ctx.check(lib.dcm_detect_interface(ctx.handle, _ptr(box_count), _ptr(s), _ptr(iface), _ptr(threshold), _ptr(g),
                                       _stream(stream)))


def dcm_remove_small_components(ctx: Context, s_in, s_out, iface, stream=None):
    ctx.check(lib.dcm_remove_small_components(ctx.handle, _ptr(s_in), _ptr(s_out), _ptr(iface), _stream(stream)))


def dcm_distance(ctx: Context, s, iface, D, iters=None, stream=None):
    ctx.check(lib.dcm_distance(ctx.handle, _ptr(s), _ptr(iface), _ptr(D), _ptr(iters), _stream(stream)))


def dcm_distance_noalloc(params: dcm_params, s, iface, D, iters=None, stream=None):
    """dcm_distance without a context or any device allocation (fixed library
    scratch); returns the status code (DCM_OK, DCM_ERR_CAPACITY, ...)."""
    return lib.dcm_distance_noalloc(ctypes.byref(params), _ptr(s), _ptr(iface), _ptr(D), _ptr(iters),
                                    _stream(stream))


def dcm_cutoffs(ctx: Context, n, pos, D, rc, stream=None):
    ctx.check(lib.dcm_cutoffs(ctx.handle, n, _ptr(pos), _ptr(D), _ptr(rc), _stream(stream)))


def dcm_forces(ctx: Context, n, pos_sorted, rc, cell_start, force, totals=None, stream=None):
    ctx.check(lib.dcm_forces(ctx.handle, n, _ptr(pos_sorted), _ptr(rc), _ptr(cell_start), _ptr(force),
                             _ptr(totals), _stream(stream)))


def dcm_set_lj(ctx: Context, eps, sigma):
    nt = len(eps)
    e = (ctypes.c_double * nt)(*[float(x) for x in eps])
    sg = (ctypes.c_double * nt)(*[float(x) for x in sigma])
    ctx.check(lib.dcm_set_lj(ctx.handle, nt, e, sg))


def dcm_forces_backward(ctx: Context, n, pos_sorted, rc, cell_start, dL_dF, dL_dE, dL_dpos, dL_dparams=None,
                        stream=None):
    ctx.check(lib.dcm_forces_backward(ctx.handle, n, _ptr(pos_sorted), _ptr(rc), _ptr(cell_start), _ptr(dL_dF),
                                      float(dL_dE), _ptr(dL_dpos), _ptr(dL_dparams), _stream(stream)))


class State:
    """Double-buffered device state for dcm_step (tensors kept alive here)."""

    def __init__(self, ctx, pos4, vel4, ids=None):
        n = pos4.shape[0]
        dev = pos4.device
        real = ctx.real
        self.n = n
        self.pos = [pos4.to(device=dev, dtype=real).contiguous(), torch.empty_like(pos4, dtype=real)]
        self.vel = [vel4.to(device=dev, dtype=real).contiguous(), torch.empty_like(vel4, dtype=real)]
        self.rc = [torch.zeros(n, dtype=real, device=dev), torch.zeros(n, dtype=real, device=dev)]
        if ids is None:
            ids = torch.arange(n, dtype=torch.int32, device=dev)
        self.id = [ids.to(device=dev, dtype=torch.int32).contiguous(), torch.empty(n, dtype=torch.int32, device=dev)]
        self.force = torch.zeros((n, 4), dtype=real, device=dev)
        self.thermo = torch.zeros(4, dtype=torch.float64, device=dev)
        self.c = dcm_state()
        for b in range(2):
            self.c.pos[b] = self.pos[b].data_ptr()
            self.c.vel[b] = self.vel[b].data_ptr()
            self.c.rc[b] = self.rc[b].data_ptr()
            self.c.id[b] = self.id[b].data_ptr()
        self.c.force = self.force.data_ptr()
        self.c.thermo = self.thermo.data_ptr()
        self.c.cur = 0
        self.c.t = 0

    @property
    def cur(self):
        return self.c.cur

    def current(self):
        k = self.c.cur
        return self.pos[k], self.vel[k], self.rc[k], self.id[k]


def dcm_step_init(ctx: Context, st: State, stream=None):
    ctx.check(lib.dcm_step_init(ctx.handle, ctypes.byref(st.c), st.n, _stream(stream)))


def dcm_step(ctx: Context, st: State, dt: float, nsteps: int = 1, stream=None):
    ctx.check(lib.dcm_step(ctx.handle, ctypes.byref(st.c), st.n, float(dt), int(nsteps), _stream(stream)))


def to_real4(xyz, w=None, dtype=torch.float32, device="cuda"):
    """(n, 3) coordinates plus an optional per-particle w (type) -> (n, 4) tensor."""
    xyz = torch.as_tensor(xyz)
    n = xyz.shape[0]
    out = torch.zeros((n, 4), dtype=dtype)
    out[:, :3] = xyz.to(dtype)
    if w is not None:
        out[:, 3] = torch.as_tensor(w).to(dtype)
    return out.to(device)


def dcm_set_timing(ctx: Context, capacity: int = 4096):
    ctx.check(lib.dcm_set_timing(ctx.handle, int(capacity)))


def dcm_stage_times(ctx: Context):
    """{stage: (ms, count)} since the last call (synchronises the device)."""
    ms = (ctypes.c_double * len(STAGES))()
    cnt = (_i64 * len(STAGES))()
    ctx.check(lib.dcm_stage_times(ctx.handle, ms, cnt))
    return {name: (ms[k], cnt[k]) for k, name in enumerate(STAGES)}


def dcm_launch_count(ctx: Context, reset: bool = False) -> int:
    c = _i64()
    ctx.check(lib.dcm_launch_count(ctx.handle, ctypes.byref(c), 1 if reset else 0))
    return c.value


def dcm_force_kernel(ctx: Context) -> int:
    k = ctypes.c_int32()
    ctx.check(lib.dcm_force_kernel(ctx.handle, ctypes.byref(k)))
    return k.value


def dcm_accumulation(ctx: Context) -> int:
    k = ctypes.c_int32()
    ctx.check(lib.dcm_accumulation(ctx.handle, ctypes.byref(k)))
    return k.value


FORCE_KERNEL_NAMES = {DCM_FORCE_THREAD: "k_forces", DCM_FORCE_PACKED: "k_forces_x2"}


# ---------------------------------------------------------------- batched form
class Batch:
    """Owns one dcm_batch: R replicas sharing params except box and size."""

    def __init__(self, params: dcm_params, boxes, counts):
        self.params = params
        self.R = len(counts)
        bx = (ctypes.c_double * (3 * self.R))(*[float(v) for b in boxes for v in b])
        cn = (_i64 * self.R)(*[int(c) for c in counts])
        h = ctypes.c_void_p()
        rc = lib.dcm_batch_create(ctypes.byref(params), self.R, bx, cn, ctypes.byref(h))
        if rc != DCM_OK:
            raise DcmError(rc, "dcm_batch_create failed")
        self.handle = h
        off = (_i64 * (self.R + 1))()
        lib.dcm_batch_offsets(h, off)
        self.offsets = list(off)
        self.n = self.offsets[-1]
        self.real = torch.float32 if params.precision == DCM_PREC_MIXED else torch.float64

    def check(self, rc):
        if rc != DCM_OK:
            raise DcmError(rc, lib.dcm_batch_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            lib.dcm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchState(State):
    """Concatenated double-buffered state of a Batch; thermo has 4 R entries."""

    def __init__(self, batch: Batch, pos4, vel4, ids=None):
        super().__init__(batch, pos4, vel4, ids)
        self.thermo = torch.zeros(4 * batch.R, dtype=torch.float64, device=pos4.device)
        self.c.thermo = self.thermo.data_ptr()


def dcm_batch_set_force_block(b: Batch, threads: int):
    b.check(lib.dcm_batch_set_force_block(b.handle, int(threads)))


def dcm_batch_step_init(b: Batch, st: BatchState, stream=None):
    b.check(lib.dcm_batch_step_init(b.handle, ctypes.byref(st.c), _stream(stream)))


def dcm_batch_step(b: Batch, st: BatchState, dt: float, nsteps: int = 1, stream=None):
    b.check(lib.dcm_batch_step(b.handle, ctypes.byref(st.c), float(dt), int(nsteps), _stream(stream)))


def dcm_batch_capture(b: Batch, st: BatchState, dt: float, stream):
    b.check(lib.dcm_batch_capture(b.handle, ctypes.byref(st.c), float(dt), _stream(stream)))


def dcm_batch_replay(b: Batch, st: BatchState, ngraphs: int, stream):
    b.check(lib.dcm_batch_replay(b.handle, ctypes.byref(st.c), int(ngraphs), _stream(stream)))


def dcm_batch_set_persistent(b: Batch, on: bool):
    b.check(lib.dcm_batch_set_persistent(b.handle, 1 if on else 0))


def dcm_batch_accumulation(b: Batch) -> int:
    k = ctypes.c_int32()
    b.check(lib.dcm_batch_accumulation(b.handle, ctypes.byref(k)))
    return k.value


def dcm_batch_set_tile(b: Batch, particles: int):
    b.check(lib.dcm_batch_set_tile(b.handle, int(particles)))


def dcm_batch_set_wait_budget(b: Batch, ns: int):
    b.check(lib.dcm_batch_set_wait_budget(b.handle, int(ns)))


def dcm_batch_barrier_selftest(b: Batch, phantom: int, budget_ns: int, stream=None) -> int:
    """Runs the persistent grid's barrier against `phantom` missing blocks;
    returns the device status (DCM_ERR_TIMEOUT when the bounded waits ran out)."""
    return lib.dcm_batch_barrier_selftest(b.handle, int(phantom), int(budget_ns), _stream(stream))


def dcm_scan_wait_selftest(ctx: Context, stream=None) -> int:
    """Runs the cell-count scan with a predecessor tile that never publishes;
    returns the device status (DCM_ERR_TIMEOUT when the bounded wait ran out)."""
    return lib.dcm_scan_wait_selftest(ctx.handle, _stream(stream))


def dcm_batch_graph_steps(b: Batch) -> int:
    return lib.dcm_batch_graph_steps(b.handle)


def dcm_batch_status(b: Batch, stream=None):
    return lib.dcm_batch_status(b.handle, _stream(stream))


def dcm_batch_set_timing(b: Batch, capacity: int = 4096):
    b.check(lib.dcm_batch_set_timing(b.handle, int(capacity)))


def dcm_batch_stage_times(b: Batch):
    ms = (ctypes.c_double * len(STAGES))()
    cnt = (_i64 * len(STAGES))()
    b.check(lib.dcm_batch_stage_times(b.handle, ms, cnt))
    return {name: (ms[k], cnt[k]) for k, name in enumerate(STAGES)}


def dcm_batch_launch_count(b: Batch, reset: bool = False) -> int:
    c = _i64()
    b.check(lib.dcm_batch_launch_count(b.handle, ctypes.byref(c), 1 if reset else 0))
    return c.value
