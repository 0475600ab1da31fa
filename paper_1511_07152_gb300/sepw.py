"""Thin ctypes binding of libsepw (include/sepw.h).

Argument marshalling only: every step of gridding, degridding, tap generation,
location, binning and the image step runs in the CUDA library.  Tensors are
torch CUDA tensors (torch provides device memory and streams); their raw
pointers and the current stream are passed through the C ABI.  If the shared
library is missing or cannot be loaded, importing this module raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

FORM_PLAIN = 0
FORM_TILED = 1
FORM_TC_BF16 = 2
FORM_TC_FP16 = 3
FORM_TC_FP16X2 = 4
FORM_TC_BF16X2 = 5
FORM_TC_TF32 = 6
GRID_TO_IMAGE = 0
IMAGE_TO_GRID = 1
IMAGE_TO_GRID_ADJOINT = 2

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP, ENOPLAN, ETOOLARGE = 0, -1, -2, -3, -4, -5, -6, -7
EBOUNDS = -8
NOALLOC_MAX_VIS = 524288
NOALLOC_MAX_TILES = 65536


class SepwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sepw error {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of struct sepw_params."""
    _fields_ = [
        ("grid_size", ctypes.c_int32),
        ("support", ctypes.c_int32),
        ("oversample", ctypes.c_int32),
        ("n_wplanes", ctypes.c_int32),
        ("fov", ctypes.c_double),
        ("w_max", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("kb_beta", ctypes.c_double),
        ("tile", ctypes.c_int32),
        ("form", ctypes.c_int32),
    ]


def make_params(grid_size, fov, support, oversample, n_wplanes, w_max,
                gamma=5.0 / 24.0, kb_beta=None, tile=0, form=FORM_TILED) -> Params:
    if kb_beta is None:
        kb_beta = 2.34 * support
    return Params(int(grid_size), int(support), int(oversample), int(n_wplanes),
                  float(fov), float(w_max), float(gamma), float(kb_beta), int(tile),
                  int(form))


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIG = {
    "sepw_version": (ctypes.c_int, []),
    "sepw_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sepw_check_params": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "sepw_taps_count": (ctypes.c_size_t, [ctypes.POINTER(Params)]),
    "sepw_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(Params)]),
    "sepw_destroy": (None, [_P]),
    "sepw_last_error": (ctypes.c_char_p, [_P]),
    "sepw_make_taps": (ctypes.c_int, [_P, _P, _P]),
    "sepw_make_taps_f64": (ctypes.c_int, [_P, _P, _P]),
    "sepw_locate": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sepw_plan": (ctypes.c_int, [_P, _I64, _P, _P, _P, _P]),
    "sepw_plan_dropped": (ctypes.c_int, [_P, ctypes.POINTER(_I64), _P]),
    "sepw_grid": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sepw_grid_planned": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "sepw_degrid": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sepw_degrid_planned": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "sepw_image": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "sepw_device_status": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), _P]),
    "sepw_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "sepw_test_stall_mma": (ctypes.c_int, [_P, ctypes.c_int]),
    "sepw_fma_probe": (ctypes.c_int, [ctypes.c_int, _I64, _P, _I64, ctypes.POINTER(_I64), _P]),
    "sepw_checked_build": (ctypes.c_int, []),
    "sepw_test_corrupt_plan": (ctypes.c_int, [_P, ctypes.c_int, _I64, ctypes.c_int32]),
    "sepw_set_schedule": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "sepw_plan_batched": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, _P]),
    "sepw_grid_batched": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P,
                                         _P, _P]),
    "sepw_grid_noalloc": (ctypes.c_int, [ctypes.POINTER(Params), _P, _I64, _P, _P, _P, _P,
                                         _P, _P, _P, _P]),
    "sepw_taper": (ctypes.c_int, [_P, _P, _P]),
    "sepw_residual_count": (ctypes.c_size_t, [ctypes.POINTER(Params), ctypes.c_int32,
                                              ctypes.c_int32]),
    "sepw_make_residual": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "sepw_make_residual_f64": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "sepw_grid_residual_planned": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                                  _P, _P, _P]),
    "sepw_degrid_residual_planned": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P,
                                                    _P, _P, _P, _P]),
    "sepw_set_facet": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "sepw_facet_shift": (ctypes.c_int, [_P, ctypes.c_int, _I64, _P, _P, _P, _P, _P, _P, _P,
                                        _P]),
    "sepw_wstack_plan": (ctypes.c_int, [_P, ctypes.c_int32, _P, _I64, _P, _P, _P, _P, _P]),
    "sepw_wstack_image": (ctypes.c_int, [_P, _P, _P, _P]),
    "sepw_wstack_model_grids": (ctypes.c_int, [_P, _P, _P, _P]),
}


def _load():
    # SEPW_CHECKED=1: the bounds-checked build (build.build(checked=True))
    checked = os.environ.get("SEPW_CHECKED", "0") not in ("", "0")
    path = _build.LIB_CHECKED if checked else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} is not built ({path}); run "
                          "paper_1511_07152_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIG.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()


def exported_symbols():
    return sorted(_SIG)


# ---- helpers ---------------------------------------------------------------


def _ptr(t, dtype=None, n=None, name="tensor"):
    """Raw device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """Owns a sepw_ctx (created on the current CUDA device)."""

    def __init__(self, params: Params):
        self.params = params
        h = _P()
        rc = LIB.sepw_create(ctypes.byref(h), ctypes.byref(params))
        if rc != OK:
            raise SepwError(rc, LIB.sepw_strerror(rc).decode())
        self.handle = h
        self.plan_nvis = 0
        self.plan_ngrids = 0
        self.wstack_nslices = 0
        self.facet = None  # (l0, m0) in facet mode

    def close(self):
        if getattr(self, "handle", None):
            LIB.sepw_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc: int):
        if rc != OK:
            msg = LIB.sepw_last_error(self.handle).decode()
            raise SepwError(rc, f"{LIB.sepw_strerror(rc).decode()}: {msg}")

    @property
    def ntaps(self) -> int:
        n = int(LIB.sepw_taps_count(ctypes.byref(self.params)))
        return 2 * n if getattr(self, "facet", None) else n

    @property
    def taps_shape(self):
        p = self.params
        shape = (p.n_wplanes, p.oversample, p.support)
        return (2,) + shape if getattr(self, "facet", None) else shape


# ---- entry points (same names as the C ABI) ---------------------------------


def sepw_version() -> int:
    return LIB.sepw_version()


def sepw_check_params(params: Params) -> int:
    return LIB.sepw_check_params(ctypes.byref(params))


def sepw_create(params: Params) -> Context:
    return Context(params)


def sepw_make_taps(ctx: Context, taps=None, stream=None):
    """complex64 taps [P, OS, S] (Eq. gt), computed in float64 on the GPU."""
    import torch
    if taps is None:
        taps = torch.empty(ctx.taps_shape, dtype=torch.complex64, device="cuda")
    ctx.check(LIB.sepw_make_taps(ctx.handle, _ptr(taps, torch.complex64, ctx.ntaps, "taps"),
                                 _stream(stream)))
    return taps


def sepw_make_taps_f64(ctx: Context, taps=None, stream=None):
    import torch
    if taps is None:
        taps = torch.empty(ctx.taps_shape, dtype=torch.complex128, device="cuda")
    ctx.check(LIB.sepw_make_taps_f64(ctx.handle,
                                     _ptr(taps, torch.complex128, ctx.ntaps, "taps"),
                                     _stream(stream)))
    return taps


def sepw_locate(ctx: Context, u, v, w, stream=None):
    import torch
    n = u.numel()
    dev = u.device
    out = dict(cu=torch.empty(n, dtype=torch.int32, device=dev),
               cv=torch.empty(n, dtype=torch.int32, device=dev),
               ou=torch.empty(n, dtype=torch.int32, device=dev),
               ov=torch.empty(n, dtype=torch.int32, device=dev),
               plane=torch.empty(n, dtype=torch.int32, device=dev),
               conj=torch.empty(n, dtype=torch.uint8, device=dev),
               keep=torch.empty(n, dtype=torch.uint8, device=dev))
    ctx.check(LIB.sepw_locate(ctx.handle, n, _ptr(u, torch.float64, n, "u"),
                              _ptr(v, torch.float64, n, "v"), _ptr(w, torch.float64, n, "w"),
                              *[out[k].data_ptr() for k in
                                ("cu", "cv", "ou", "ov", "plane", "conj", "keep")],
                              _stream(stream)))
    return out


def sepw_plan(ctx: Context, u, v, w, stream=None):
    import torch
    n = u.numel()
    ctx.check(LIB.sepw_plan(ctx.handle, n, _ptr(u, torch.float64, n, "u"),
                            _ptr(v, torch.float64, n, "v"), _ptr(w, torch.float64, n, "w"),
                            _stream(stream)))
    ctx.plan_nvis = n
    ctx.plan_ngrids = 1


def _offsets(offsets):
    import numpy as np
    o = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if o.ndim != 1 or o.size < 2:
        raise ValueError("vis_offsets must be 1-D with ngrids + 1 entries")
    return o


def sepw_plan_batched(ctx: Context, vis_offsets, u, v, w, stream=None):
    """Plan ngrids = len(vis_offsets) - 1 grids in one work list (host
    offsets, copied during the call)."""
    import torch
    o = _offsets(vis_offsets)
    n = u.numel()
    if int(o[-1]) != n:
        raise ValueError("vis_offsets[-1] must equal the number of visibilities")
    ctx.check(LIB.sepw_plan_batched(ctx.handle, o.size - 1, o.ctypes.data,
                                    _ptr(u, torch.float64, n, "u"),
                                    _ptr(v, torch.float64, n, "v"),
                                    _ptr(w, torch.float64, n, "w"), _stream(stream)))
    ctx.plan_nvis = n
    ctx.plan_ngrids = o.size - 1


def sepw_grid_batched(ctx: Context, taps, vis_offsets, u, v, w, vis, weight, grids,
                      n_dropped=None, stream=None):
    import torch
    o = _offsets(vis_offsets)
    n = u.numel()
    N = ctx.params.grid_size
    ng = o.size - 1
    ctx.check(LIB.sepw_grid_batched(ctx.handle, _ptr(taps, torch.complex64, ctx.ntaps, "taps"),
                                    ng, o.ctypes.data, _ptr(u, torch.float64, n, "u"),
                                    _ptr(v, torch.float64, n, "v"),
                                    _ptr(w, torch.float64, n, "w"),
                                    _ptr(vis, torch.complex64, n, "vis"),
                                    _ptr(weight, torch.float32, n, "weight"),
                                    _ptr(grids, torch.complex64, ng * N * N, "grids"),
                                    _ptr(n_dropped, torch.int64, 1, "n_dropped"),
                                    _stream(stream)))
    ctx.plan_nvis = n
    ctx.plan_ngrids = ng
    return grids


def sepw_plan_dropped(ctx: Context, stream=None) -> int:
    out = _I64(0)
    ctx.check(LIB.sepw_plan_dropped(ctx.handle, ctypes.byref(out), _stream(stream)))
    return int(out.value)


def sepw_grid(ctx: Context, taps, u, v, w, vis, weight, grid, n_dropped=None, stream=None):
    import torch
    n = u.numel()
    N = ctx.params.grid_size
    ctx.check(LIB.sepw_grid(ctx.handle, _ptr(taps, torch.complex64, ctx.ntaps, "taps"), n,
                            _ptr(u, torch.float64, n, "u"), _ptr(v, torch.float64, n, "v"),
                            _ptr(w, torch.float64, n, "w"),
                            _ptr(vis, torch.complex64, n, "vis"),
                            _ptr(weight, torch.float32, n, "weight"),
                            _ptr(grid, torch.complex64, N * N, "grid"),
                            _ptr(n_dropped, torch.int64, 1, "n_dropped"), _stream(stream)))
    ctx.plan_nvis = n
    ctx.plan_ngrids = 1
    return grid


def sepw_grid_planned(ctx: Context, taps, vis, weight, grid, stream=None):
    import torch
    n = ctx.plan_nvis
    N = ctx.params.grid_size * ctx.params.grid_size * getattr(ctx, "plan_ngrids", 1)
    ctx.check(LIB.sepw_grid_planned(ctx.handle, _ptr(taps, torch.complex64, ctx.ntaps, "taps"),
                                    _ptr(vis, torch.complex64, n, "vis"),
                                    _ptr(weight, torch.float32, n, "weight"),
                                    _ptr(grid, torch.complex64, N, "grid"),
                                    _stream(stream)))
    return grid


def sepw_degrid(ctx: Context, taps, u, v, w, grid, weight, vis_out, n_dropped=None,
                stream=None):
    import torch
    n = u.numel()
    N = ctx.params.grid_size
    ctx.check(LIB.sepw_degrid(ctx.handle, _ptr(taps, torch.complex64, ctx.ntaps, "taps"), n,
                              _ptr(u, torch.float64, n, "u"), _ptr(v, torch.float64, n, "v"),
                              _ptr(w, torch.float64, n, "w"),
                              _ptr(grid, torch.complex64, N * N, "grid"),
                              _ptr(weight, torch.float32, n, "weight"),
                              _ptr(vis_out, torch.complex64, n, "vis_out"),
                              _ptr(n_dropped, torch.int64, 1, "n_dropped"), _stream(stream)))
    ctx.plan_nvis = n
    ctx.plan_ngrids = 1
    return vis_out


def sepw_degrid_planned(ctx: Context, taps, grid, weight, vis_out, stream=None):
    import torch
    n = ctx.plan_nvis
    N = ctx.params.grid_size * ctx.params.grid_size * getattr(ctx, "plan_ngrids", 1)
    ctx.check(LIB.sepw_degrid_planned(ctx.handle,
                                      _ptr(taps, torch.complex64, ctx.ntaps, "taps"),
                                      _ptr(grid, torch.complex64, N, "grid"),
                                      _ptr(weight, torch.float32, n, "weight"),
                                      _ptr(vis_out, torch.complex64, n, "vis_out"),
                                      _stream(stream)))
    return vis_out


def sepw_device_status(ctx: Context, stream=None) -> int:
    """Status recorded by the context's kernels (OK or ETIMEOUT); resets it."""
    st = ctypes.c_int(0)
    ctx.check(LIB.sepw_device_status(ctx.handle, ctypes.byref(st), _stream(stream)))
    return int(st.value)


def sepw_set_wait_limit(ctx: Context, limit_ns: int):
    """Limit of every bounded wait in the context's tensor-core kernels."""
    ctx.check(LIB.sepw_set_wait_limit(ctx.handle, int(limit_ns)))


def sepw_set_schedule(ctx: Context, chunk: int = 0, grid_parts: int = 0):
    """Work-item size and block-gridder parts of the next plans (0: defaults)."""
    ctx.check(LIB.sepw_set_schedule(ctx.handle, int(chunk), int(grid_parts)))
    ctx.plan_nvis = 0


def sepw_test_stall_mma(ctx: Context, enable: bool):
    """Test hook: the tensor-core kernels issue no MMAs, so their waits run out."""
    ctx.check(LIB.sepw_test_stall_mma(ctx.handle, 1 if enable else 0))


def sepw_fma_probe(paired: bool, iters: int, out, stream=None) -> int:
    """Launch the FP32 FMA rate probe on `stream` (scalar FFMA, or paired
    FFMA2 when `paired`); `out` is a float32 CUDA tensor of at least
    SMs x 1024 elements.  Returns the launch's flop count; the caller times
    the launch with CUDA events."""
    import torch
    flops = _I64(0)
    rc = LIB.sepw_fma_probe(1 if paired else 0, int(iters),
                            _ptr(out, torch.float32, out.numel(), "out"), int(out.numel()),
                            ctypes.byref(flops), _stream(stream))
    if rc != OK:
        raise SepwError(rc, "sepw_fma_probe")
    return int(flops.value)


def sepw_checked_build() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return LIB.sepw_checked_build() != 0


def sepw_test_corrupt_plan(ctx: Context, which: int, slot: int, value: int):
    """Test hook of the checked build: overwrite the plan's slot -> visibility
    index (which = 0) or a record's plane field (which = 1) at `slot`."""
    ctx.check(LIB.sepw_test_corrupt_plan(ctx.handle, int(which), int(slot), int(value)))


def sepw_image(ctx: Context, direction: int, buf, stream=None):
    import torch
    N = ctx.params.grid_size
    ctx.check(LIB.sepw_image(ctx.handle, int(direction),
                             _ptr(buf, torch.complex64, N * N, "buf"), _stream(stream)))
    return buf


def _residual_shape(ctx: Context, support_r, oversample_r):
    p = ctx.params
    n = int(LIB.sepw_residual_count(ctypes.byref(p), int(support_r), int(oversample_r)))
    if n == 0:
        raise SepwError(EINVAL, "invalid correction table sizes")
    return (p.n_wplanes, oversample_r, oversample_r, support_r, support_r), n


def sepw_make_residual(ctx: Context, support_r, oversample_r, table=None, stream=None):
    """Correction table F_w - F~_w, complex64 [P, OSr, OSr, Sr, Sr] (Sec. 7)."""
    import torch
    shape, n = _residual_shape(ctx, support_r, oversample_r)
    if table is None:
        table = torch.empty(shape, dtype=torch.complex64, device="cuda")
    ctx.check(LIB.sepw_make_residual(ctx.handle, int(support_r), int(oversample_r),
                                     _ptr(table, torch.complex64, n, "table"), _stream(stream)))
    return table


def sepw_make_residual_f64(ctx: Context, support_r, oversample_r, table=None, stream=None):
    import torch
    shape, n = _residual_shape(ctx, support_r, oversample_r)
    if table is None:
        table = torch.empty(shape, dtype=torch.complex128, device="cuda")
    ctx.check(LIB.sepw_make_residual_f64(ctx.handle, int(support_r), int(oversample_r),
                                         _ptr(table, torch.complex128, n, "table"),
                                         _stream(stream)))
    return table


def sepw_grid_residual_planned(ctx: Context, table, vis, weight, grid, stream=None):
    """Correction pass: adds the correction table's update to grid."""
    import torch
    Sr, OSr = int(table.shape[-1]), int(table.shape[1])
    N = ctx.params.grid_size
    n = ctx.plan_nvis
    ctx.check(LIB.sepw_grid_residual_planned(
        ctx.handle, Sr, OSr, _ptr(table, torch.complex64, table.numel(), "table"),
        _ptr(vis, torch.complex64, n, "vis"), _ptr(weight, torch.float32, n, "weight"),
        _ptr(grid, torch.complex64, ctx.plan_ngrids * N * N, "grid"), _stream(stream)))
    return grid


def sepw_degrid_residual_planned(ctx: Context, table, grid, weight, vis_out, stream=None):
    """Adjoint of the correction pass: adds to vis_out."""
    import torch
    Sr, OSr = int(table.shape[-1]), int(table.shape[1])
    N = ctx.params.grid_size
    n = ctx.plan_nvis
    ctx.check(LIB.sepw_degrid_residual_planned(
        ctx.handle, Sr, OSr, _ptr(table, torch.complex64, table.numel(), "table"),
        _ptr(grid, torch.complex64, ctx.plan_ngrids * N * N, "grid"),
        _ptr(weight, torch.float32, n, "weight"), _ptr(vis_out, torch.complex64, n, "vis_out"),
        _stream(stream)))
    return vis_out


FACET_IN, FACET_OUT = 0, 1


def sepw_set_facet(ctx: Context, l0=None, m0=None):
    """Facet mode for the facet centred at (l0, m0) (Sec. 4.1); None leaves
    it.  In facet mode the taps are two tables [2, P, OS, S]."""
    if l0 is None:
        ctx.check(LIB.sepw_set_facet(ctx.handle, 0, 0.0, 0.0))
        ctx.facet = None
    else:
        ctx.check(LIB.sepw_set_facet(ctx.handle, 1, float(l0), float(m0)))
        ctx.facet = (float(l0), float(m0))


def sepw_facet_shift(ctx: Context, direction, u, v, w, vis=None, u_out=None, v_out=None,
                     vis_out=None, stream=None):
    """Visibilities into (FACET_IN) or out of (FACET_OUT) the context's facet."""
    import torch
    n = u.numel()
    ctx.check(LIB.sepw_facet_shift(ctx.handle, int(direction), n,
                                   _ptr(u, torch.float64, n, "u"),
                                   _ptr(v, torch.float64, n, "v"),
                                   _ptr(w, torch.float64, n, "w"),
                                   _ptr(vis, torch.complex64, n, "vis"),
                                   _ptr(u_out, torch.float64, n, "u_out"),
                                   _ptr(v_out, torch.float64, n, "v_out"),
                                   _ptr(vis_out, torch.complex64, n, "vis_out"),
                                   _stream(stream)))


def sepw_taper(ctx: Context, out=None, stream=None):
    """c1(nu_a), a = 0..N-1 (float32, device)."""
    import torch
    N = ctx.params.grid_size
    if out is None:
        out = torch.empty(N, dtype=torch.float32, device=torch.cuda.current_device())
    ctx.check(LIB.sepw_taper(ctx.handle, _ptr(out, torch.float32, N, "taper"), _stream(stream)))
    return out


def sepw_wstack_plan(ctx: Context, w_centres, u, v, w, slice_out=None, stream=None):
    """Hybrid W-stacking plan (slices at the host centres w_centres); the
    context's plan then grids / degrids len(w_centres) grids with the
    visibilities in the caller's order."""
    import numpy as np
    import torch
    c = np.ascontiguousarray(np.asarray(w_centres, np.float64))
    n = u.numel()
    ctx.check(LIB.sepw_wstack_plan(ctx.handle, int(c.size), c.ctypes.data, n,
                                   _ptr(u, torch.float64, n, "u"),
                                   _ptr(v, torch.float64, n, "v"),
                                   _ptr(w, torch.float64, n, "w"),
                                   _ptr(slice_out, torch.int32, n, "slice_out"),
                                   _stream(stream)))
    ctx.plan_nvis = n
    ctx.plan_ngrids = int(c.size)
    ctx.wstack_nslices = int(c.size)


def sepw_wstack_image(ctx: Context, slice_grids, image, stream=None):
    """Dirty image from the slice grids (transformed in place)."""
    import torch
    N = ctx.params.grid_size
    L = ctx.wstack_nslices
    ctx.check(LIB.sepw_wstack_image(ctx.handle,
                                    _ptr(slice_grids, torch.complex64, L * N * N, "slice_grids"),
                                    _ptr(image, torch.complex64, N * N, "image"),
                                    _stream(stream)))
    return image


def sepw_wstack_model_grids(ctx: Context, image, slice_grids, stream=None):
    """Slice grids of a model image for W-stacking prediction."""
    import torch
    N = ctx.params.grid_size
    L = ctx.wstack_nslices
    ctx.check(LIB.sepw_wstack_model_grids(ctx.handle,
                                          _ptr(image, torch.complex64, N * N, "image"),
                                          _ptr(slice_grids, torch.complex64, L * N * N,
                                               "slice_grids"),
                                          _stream(stream)))
    return slice_grids


def sepw_grid_noalloc(params: Params, taps, u, v, w, vis, weight, grid, n_dropped=None,
                      stream=None) -> int:
    """Gridding without any device allocation (fixed scratch compiled into the
    library).  Returns the status code instead of raising, so a caller can see
    SEPW_ETOOLARGE."""
    import torch
    n = u.numel()
    N = params.grid_size
    ntaps = params.n_wplanes * params.oversample * params.support
    return int(LIB.sepw_grid_noalloc(ctypes.byref(params),
                                     _ptr(taps, torch.complex64, ntaps, "taps"), n,
                                     _ptr(u, torch.float64, n, "u"),
                                     _ptr(v, torch.float64, n, "v"),
                                     _ptr(w, torch.float64, n, "w"),
                                     _ptr(vis, torch.complex64, n, "vis"),
                                     _ptr(weight, torch.float32, n, "weight"),
                                     _ptr(grid, torch.complex64, N * N, "grid"),
                                     _ptr(n_dropped, torch.int64, 1, "n_dropped"),
                                     _stream(stream)))
