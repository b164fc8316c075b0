"""The C-ABI library builds, loads and exports every symbol include/dcm.h
declares; host-only entry points behave as documented (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dcm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s+\**(dcm_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1701_05242_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("dcm_bin", "dcm_detect_interface", "dcm_distance", "dcm_cutoffs", "dcm_forces", "dcm_step",
                     "dcm_create", "dcm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    src = open(os.path.join(ROOT, "paper_1701_05242_gb300", "dcm.py")).read()
    for n in declared_functions():
        assert f'"{n}"' in src, n


def _params(lib, **kw):
    import paper_1701_05242_gb300.dcm as D  # noqa: F401  (loads the library; no GPU call)
    p = D.make_params(kw.pop("box", (12.0, 12.0, 48.0)), **kw)
    return D, p


def test_params_default_and_validate(lib):
    D, p = _params(lib)
    assert p.h == 1.5 and p.l == 1.5 and p.rc_min == 3.0 and p.rc_max == 6.0 and p.smooth_w == 2
    assert p.precision == D.DCM_PREC_MIXED and p.recompute_every == 10 and p.threshold == -1
    assert p.accumulation == D.DCM_ACC_AUTO
    rc, msg = D.dcm_validate_params(p)
    assert rc == D.DCM_OK, msg


@pytest.mark.parametrize("kw,code", [
    (dict(box=(12.0, 12.0, 47.0)), 2),          # not a multiple of l
    (dict(l=1.3), 2),                           # long mantissa edge
    (dict(rc_max=6.5), 2),                      # rc_max > L/2 of the 12-box
    (dict(rc_min=4.0, rc_max=3.0), 1),
    (dict(ntypes=5), 1),
    (dict(iter_max=0), 1),
    (dict(recompute_every=0), 1),
    (dict(precision=7), 1),
    (dict(n_max=-1), 1),
    (dict(n_max=2 ** 31), 1),
    (dict(box=(4000.5, 4000.5, 4000.5)), 2),    # each axis < 65536 cells, 2^31 or more in all
    (dict(box=(99000.0, 12.0, 48.0)), 2),       # 66000 cells along x
    (dict(min_component=-1), 1),
    (dict(force_kernel=9), 1),
    (dict(force_kernel=2), 1),                  # removed kernel numbers stay invalid
    (dict(force_kernel=5), 1),
    (dict(accumulation=8), 1),
    (dict(newton3=1), 1),                       # Newton's third law form needs Verlet lists
    (dict(newton3=2, skin=0.3, rc_max=5.5), 1),
    (dict(accumulation=-1), 1),
    (dict(skin=-0.1), 1),
    (dict(skin=0.5, rc_max=5.8), 2),             # rc_max + skin > L/2
    (dict(skin=0.3, rc_max=5.5, n_max=2 ** 26), 5),  # list entries keep 26 index bits
    (dict(lx=-0.75), 1),
    (dict(lx=1.3), 2),                          # long mantissa
    (dict(lx=0.625), 2),                        # 12 / 0.625 is not an integer
])
def test_params_rejected(lib, kw, code):
    D, p = _params(lib, **kw)
    rc, msg = D.dcm_validate_params(p)
    assert rc == code and msg


def test_grid_dims_and_scratch(lib):
    D, p = _params(lib, box=(240.0, 240.0, 960.0), n_max=15482880)
    cells = (ctypes.c_int64 * 3)()
    boxes = (ctypes.c_int64 * 3)()
    assert D.lib.dcm_grid_dims(ctypes.byref(p), cells, boxes) == 0
    assert tuple(cells) == (160, 160, 640) and tuple(boxes) == (160, 160, 640)
    D, p = _params(lib, box=(240.0, 240.0, 960.0), n_max=15482880, lx=0.75)
    assert D.lib.dcm_grid_dims(ctypes.byref(p), cells, boxes) == 0
    assert tuple(cells) == (320, 160, 640) and tuple(boxes) == (160, 160, 640)
    b = ctypes.c_int64()
    assert D.lib.dcm_scratch_bytes(ctypes.byref(p), ctypes.byref(b)) == 0
    assert 0.2e9 < b.value < 2e9
    assert b"sm_103a" in D.lib.dcm_version()


def test_tensors_must_be_on_device(lib):
    import torch
    D, _ = _params(lib)
    with pytest.raises(ValueError):
        D._ptr(torch.zeros(4))
