"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/sepw.h declares, and validates parameters on the host."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sepw.h")


@pytest.fixture(scope="module")
def sepw():
    from paper_1511_07152_gb300 import build
    build.build()
    import paper_1511_07152_gb300.sepw as S
    return S


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"SEPW_API\s+[^;(]*?\b(sepw_\w+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("sepw_make_taps", "sepw_grid", "sepw_degrid", "sepw_image", "sepw_locate",
                 "sepw_plan", "sepw_create", "sepw_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(sepw):
    lib = ctypes.CDLL(sepw.LIB._name)
    for name in _declared():
        assert hasattr(lib, name), name
    # and the binding wraps exactly those
    assert sorted(sepw.exported_symbols()) == _declared()


def test_version(sepw):
    assert sepw.sepw_version() == 1


def _p(sepw, **kw):
    base = dict(grid_size=256, fov=math.radians(2.0), support=8, oversample=8,
                n_wplanes=32, w_max=2000.0)
    base.update(kw)
    return sepw.make_params(**base)


@pytest.mark.parametrize("kw,ok", [
    ({}, True),
    (dict(grid_size=255), False),
    (dict(grid_size=8), False),
    (dict(support=7), False),
    (dict(support=34), False),
    (dict(oversample=0), False),
    (dict(oversample=257), False),
    (dict(n_wplanes=0), False),
    (dict(fov=0.0), False),
    (dict(fov=float("nan")), False),
    (dict(fov=1.5), False),
    (dict(w_max=0.0), False),
    (dict(w_max=float("inf")), False),
    (dict(kb_beta=-1.0), False),
    (dict(tile=7), False),
    (dict(tile=64, support=16), False),
    (dict(tile=48, support=16), True),
    (dict(form=99), False),
    (dict(n_wplanes=1), True),
    (dict(support=32, tile=32), True),
])
def test_check_params(sepw, kw, ok):
    rc = sepw.sepw_check_params(_p(sepw, **kw))
    assert (rc == 0) == ok
    n = sepw.LIB.sepw_taps_count(ctypes.byref(_p(sepw, **kw)))
    if ok:
        p = _p(sepw, **kw)
        assert n == p.n_wplanes * p.oversample * p.support
    else:
        assert n == 0


def test_null_arguments_rejected_without_gpu(sepw):
    L = sepw.LIB
    assert L.sepw_check_params(None) == sepw.EINVAL
    assert L.sepw_create(None, ctypes.byref(_p(sepw))) == sepw.EINVAL
    h = ctypes.c_void_p()
    assert L.sepw_create(ctypes.byref(h), ctypes.byref(_p(sepw, support=3))) == sepw.EINVAL
    assert not h.value
    L.sepw_destroy(None)  # no-op
    assert L.sepw_make_taps(None, None, None) == sepw.EINVAL
    assert L.sepw_grid(None, None, 0, None, None, None, None, None, None, None, None) == \
        sepw.EINVAL
    assert L.sepw_image(None, 0, None, None) == sepw.EINVAL
    assert L.sepw_strerror(sepw.EINVAL) == b"invalid argument"
    # the FMA probe checks its arguments before any CUDA call
    flops = ctypes.c_int64(-1)
    dummy = ctypes.c_float(0.0)
    for paired, iters in ((0, 0), (1, -5), (0, (1 << 30) + 1)):
        assert L.sepw_fma_probe(paired, iters, ctypes.byref(dummy), 1 << 20,
                                ctypes.byref(flops), None) == sepw.EINVAL
    assert L.sepw_fma_probe(0, 10, None, 1 << 20, ctypes.byref(flops), None) == sepw.EINVAL
    assert L.sepw_fma_probe(0, 10, ctypes.byref(dummy), 1 << 20, None, None) == sepw.EINVAL
    assert flops.value == -1


def test_params_struct_layout(sepw):
    """The ctypes mirror has the C layout (4 int32, 4 double, 2 int32)."""
    P = sepw.Params
    assert ctypes.sizeof(P) == 56
    assert P.fov.offset == 16 and P.kb_beta.offset == 40 and P.form.offset == 52


def test_product_path_does_not_import_oracle():
    """The CUDA path and the oracle share no code and neither imports the
    other."""
    pkg = os.path.join(ROOT, "paper_1511_07152_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "sepw_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1511_07152_gb300" not in txt, f
