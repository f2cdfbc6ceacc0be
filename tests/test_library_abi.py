"""The C ABI library builds, loads and exports every function declared in
include/stab.h; argument errors are rejected before any device work (no GPU
needed)."""
import ctypes as C
import os
import re

import pytest

from paper_1701_03572_gb300 import build as build_lib
from paper_1701_03572_gb300 import stab as S

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "stab.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stab_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    lib = C.CDLL(build_lib())
    names = declared_functions()
    assert len(names) >= 35
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_every_declared_function():
    import inspect
    src = inspect.getsource(S)
    missing = [n for n in declared_functions() if f'"{n}"' not in src]
    assert missing == []


def test_default_params_and_argument_errors_without_a_device():
    p = S.default_params()
    assert (p.max_corners, p.levels, p.win_radius, p.max_iters, p.redetect_period) == (200, 3, 10, 30, 5)
    assert abs(p.eps - 0.01) < 1e-9 and p.model == S.STAB_SIMILARITY and p.precision == S.STAB_FP32
    # the last fields line up with the library's layout (hybrid dwell, crop zoom)
    assert p.dwell == 20 and p.crop_zoom == 1.0
    assert C.sizeof(S.StabMotion) == 4 * S.MOTION_WORDS and C.sizeof(S.StabAffine) == 4 * S.AFFINE_WORDS
    L = S.lib()
    h = C.c_void_p()
    bad = [dict(max_corners=0), dict(max_corners=4096), dict(levels=0), dict(levels=9), dict(win_radius=13),
           dict(smooth_window=64), dict(model=7), dict(precision=3), dict(inlier_thresh=0.0), dict(roi_margin_x=1),
           dict(model=3), dict(dwell=0), dict(crop_zoom=0.5), dict(crop_zoom=4.5), dict(crop_zoom=float("nan"))]
    for kw in bad:
        q = S.default_params(**kw)
        assert L.stab_create(320, 240, C.byref(q), C.byref(h)) == -1, kw
        assert not h.value
    q = S.default_params(levels=8)
    assert L.stab_create(64, 64, C.byref(q), C.byref(h)) == -1          # too many levels for the size
    assert L.stab_create(8, 240, C.byref(S.default_params()), C.byref(h)) == -1
    assert L.stab_batch_create(0, None, 0, C.byref(h)) == -1
    assert L.stab_detect_noalloc(None, 100, 100, 100, 3, 3, 97, 97, 0.01, 10, None, None, None, None, None) == -1
    arr = (C.c_float * 4)()
    assert L.stab_charb_forward(arr, arr, 640, 480, 1, arr, 300, 1e-3, None, None, None, None) == -1   # margin too big
    assert L.stab_charb_forward(arr, arr, 640, 480, 1, arr, 48, 0.0, None, None, None, None) == -1     # eps <= 0
    assert L.stab_version().startswith(b"gb300-stab")


def test_variant_count_matches_the_library():
    assert S.lib().stab_lk_variants() == S.LK_VARIANTS
