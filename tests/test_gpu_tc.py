"""Tensor-core contraction form (tcgen05) of the gridder against the FP64
oracle.

The operands are rounded to BF16 (unit roundoff u = 2^-8), FP16 or TF32 (both
11-bit significands, u = 2^-11; TF32 keeps the FP32 exponent range) and
accumulated in FP32.  Every product W V F1(u) F1(v) then carries two
independent operand roundings, relative rms sqrt(2/3) u, and the grid's
relative L2 error is about that: 3.2e-3 (BF16) and 4.0e-4 (FP16, TF32).  The
bars below allow a factor ~3: 1e-2 and 1.5e-3.

The split forms represent each operand as hi + lo, hi = rn(x), lo = rn(x - hi),
and take all four products of the splits, so only the rounding of lo is left:
at most half an ulp of lo, 2^-17 of the operand for BF16 (8-bit significands)
and 2^-22 for FP16 (11 bits, after the per-item scale puts the largest |W V|
near 1).  Uniform over that interval, the product's relative rms is 3.3e-6
(BF16 hi + lo) and 1.9e-7 (FP16 hi + lo), measured on a million random
operand pairs; both forms are held to the FP32 forms' bar, 1e-5.  Degridding
in the BF16 and FP16 forms is the contraction form on tensor cores with the
same bars, and so is degridding in the hi + lo forms, whose contraction takes
three of the four products (a_lo X_lo dropped: relative rms about
(2^-8.5 / sqrt(3))^2 = 2.6e-6 (BF16) and 4e-8 (FP16) per product, on top of
the representation error above), held to 1e-5; the TF32 form degrids with
the tiled FP32 kernel.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL = {"bf16": 1e-2, "fp16": 1.5e-3, "fp16x2": 1e-5, "bf16x2": 1e-5, "tf32": 1.5e-3}
PRECS = ["bf16", "fp16", "fp16x2", "bf16x2", "tf32"]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_07152_gb300 import build
    build.build()
    import paper_1511_07152_gb300.sepw as S
    return torch, S


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _form(S, name):
    return {"bf16": S.FORM_TC_BF16, "fp16": S.FORM_TC_FP16, "fp16x2": S.FORM_TC_FP16X2,
            "bf16x2": S.FORM_TC_BF16X2, "tf32": S.FORM_TC_TF32}[name]


def _grid(torch, S, wl, form, tile=0):
    ctx = S.sepw_create(S.make_params(**wl.params(), tile=tile, form=form))
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    N = wl.grid_size
    grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    nd = torch.zeros(1, dtype=torch.int64, device="cuda")
    S.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], grid, nd)
    assert S.sepw_device_status(ctx) == S.OK
    return grid.cpu().numpy(), int(nd.item()), ctx, taps, d


def _oracle(wl):
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    return O.grid_separable(p, loc, wl.vis, wl.weight, O.taps(p)), loc


CASES = {
    "small_disk_S8": lambda: synth.small_disk(),
    "rand_S12": lambda: synth.random_case(2, 6000, 160, 12, 16, 17, edge_fraction=0.1),
    "rand_S16": lambda: synth.random_case(3, 20000, 256, 16, 16, 33, edge_fraction=0.1),
}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(CASES))
def test_tc_grid_parity(env, prec, name):
    torch, S = env
    wl = CASES[name]()
    want, loc = _oracle(wl)
    got, nd, *_ = _grid(torch, S, wl, _form(S, prec))
    err = rel_l2(got, want)
    assert err <= TOL[prec], err
    assert nd == int((~loc["keep"]).sum())


@pytest.mark.parametrize("tile", [8, 12, 16])
@pytest.mark.parametrize("prec", ["bf16", "fp16", "bf16x2", "fp16x2", "tf32"])
def test_tc_tile_sizes(env, tile, prec):
    """Tiles up to the 32-cell window (T + S - 1 <= 32 at S = 16): gridding,
    and degridding, whose first K chunk ly / 4 ranges over 0 .. (T - 1) / 4."""
    torch, S = env
    wl = CASES["rand_S16"]()
    want, loc = _oracle(wl)
    got, _, ctx, taps, d = _grid(torch, S, wl, _form(S, prec), tile=tile)
    assert rel_l2(got, want) <= TOL[prec]
    p = O.params_from(wl.params())
    N = wl.grid_size
    rng = np.random.default_rng(tile)
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    want_p = O.degrid_separable(p, loc, X, wl.weight, O.taps(p))
    out = torch.zeros(wl.nvis, dtype=torch.complex64, device="cuda")
    S.sepw_degrid(ctx, taps, d["u"], d["v"], d["w"], torch.from_numpy(X).cuda(), d["weight"], out)
    assert S.sepw_device_status(ctx) == S.OK
    assert rel_l2(out.cpu().numpy(), want_p) <= TOL[prec]


def test_tc_tile_beyond_window_rejected(env):
    torch, S = env
    wl = CASES["rand_S16"]()
    for tile in (18, 32, 48):
        assert S.sepw_check_params(S.make_params(**wl.params(), tile=tile,
                                                 form=S.FORM_TC_BF16)) == S.EINVAL
        assert S.sepw_check_params(S.make_params(**wl.params(), tile=tile,
                                                 form=S.FORM_TILED)) == S.OK


def test_tc_heavy_tile(env):
    """One position holds 50,000 visibilities: many work items and stages on
    one tile, accumulated through several epilogues."""
    torch, S = env
    n = 60000
    rng = np.random.default_rng(4)
    fov = math.radians(2.0)
    u = np.concatenate([np.full(50000, 2.2 / fov), rng.uniform(-6, 6, n - 50000) / fov])
    v = np.concatenate([np.full(50000, -3.9 / fov), rng.uniform(-6, 6, n - 50000) / fov])
    w = rng.uniform(-300, 300, n)
    vis = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    wt = rng.uniform(0.5, 1, n).astype(np.float32)
    wl = synth.Workload("heavy", 96, fov, 16, 16, 9, 300.0, u, v, w, vis, wt)
    want, _ = _oracle(wl)
    # A cell of the heavy position sums 50,000 zero-mean terms in FP32 (in an
    # order the atomics choose): rounding each growing partial sum costs
    # about 2^-24 sqrt(n / 2) = 9.4e-6 of the result, the floor of any form
    # that accumulates in FP32.  The hi + lo form's bar is three times that.
    floor = 3.0 * 2.0 ** -24 * math.sqrt(50000 / 2)
    for prec in ("fp16", "fp16x2", "bf16x2", "tf32"):
        got, *_ = _grid(torch, S, wl, _form(S, prec))
        assert rel_l2(got, want) <= max(TOL[prec], floor), prec


@pytest.mark.parametrize("amp", [1e-7, 1e6, 3e30])
@pytest.mark.parametrize("prec", ["fp16", "fp16x2", "bf16x2", "tf32"])
def test_tc_fp16_amplitude_range(env, amp, prec):
    """Visibility amplitudes far outside FP16's range: the per-item
    power-of-two scale keeps the FP16 operands representable, BF16 and TF32
    have the FP32 exponent range, and the error bar is unchanged (the grid scales
    with the amplitude)."""
    torch, S = env
    wl = CASES["rand_S16"]()
    wl.vis = (wl.vis.astype(np.complex128) * amp).astype(np.complex64)
    want, _ = _oracle(wl)
    got, *_ = _grid(torch, S, wl, _form(S, prec))
    assert np.all(np.isfinite(got))
    assert rel_l2(got, want) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(CASES))
def test_tc_degrid_parity(env, prec, name):
    """Degridding in the tensor-core forms: the contraction form
    Q = conj(Av) X per window for BF16, FP16 and their hi + lo splits (bars
    as for gridding: each product carries the same two operand roundings),
    the tiled FP32 kernel for TF32.  Dropped visibilities get 0."""
    torch, S = env
    wl = CASES[name]()
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    N = wl.grid_size
    rng = np.random.default_rng(8)
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    want = O.degrid_separable(p, loc, X, wl.weight, O.taps(p))
    _, _, ctx, taps, d = _grid(torch, S, wl, _form(S, prec))
    out = torch.full((wl.nvis,), complex(3, 3), dtype=torch.complex64, device="cuda")
    S.sepw_degrid(ctx, taps, d["u"], d["v"], d["w"], torch.from_numpy(X).cuda(),
                  d["weight"], out)
    assert S.sepw_device_status(ctx) == S.OK
    got = out.cpu().numpy()
    assert rel_l2(got, want) <= TOL[prec]
    assert np.all(got[~loc["keep"]] == 0)


@pytest.mark.parametrize("prec", ["fp16", "fp16x2"])
@pytest.mark.parametrize("amp", [1e-7, 1e6, 3e30])
def test_tc_degrid_fp16_amplitude_range(env, amp, prec):
    """Model grids far outside FP16's range: the per-item scale of the window
    keeps the operands (both parts of the split form) representable."""
    torch, S = env
    wl = CASES["rand_S16"]()
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    N = wl.grid_size
    rng = np.random.default_rng(9)
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) * amp
    want = O.degrid_separable(p, loc, X, wl.weight, O.taps(p))
    _, _, ctx, taps, d = _grid(torch, S, wl, _form(S, prec))
    out = torch.empty(wl.nvis, dtype=torch.complex64, device="cuda")
    S.sepw_degrid(ctx, taps, d["u"], d["v"], d["w"],
                  torch.from_numpy(X.astype(np.complex64)).cuda(), d["weight"], out)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert rel_l2(got, want) <= TOL[prec]


def _round_fp16(a):
    """Round to an 11-bit significand at any exponent: FP16 after the
    kernel's power-of-two scale, with the subnormal range left out."""
    m, e = np.frexp(a)
    return np.ldexp(np.round(m * 2048.0) / 2048.0, e)


def test_tc_degrid_fp16_error_follows_operand_rounding(env):
    """FP16 degridding errs relative to the model grid, not to the
    prediction.  A white image through IMAGE_TO_GRID (divided by n c1 c1)
    gives a grid whose rms is ~500 times the prediction's, since degridding
    (whose image-domain response is c1 c1) cancels the edge-amplified part;
    11-bit operands then cost ~3% of the prediction.  The kernel's error
    equals that of the same degridding in FP64 on operands rounded to 11
    bits (grid and taps), to within 10%."""
    torch, S = env
    wl = synth.random_case(42, 6000, 128, 8, 8, 9, w_max=300.0, radius_cells=50.0)
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    T = O.taps(p)
    image = np.random.default_rng(3).standard_normal((128, 128))
    X = O.image_to_grid(p, image)
    want = O.degrid_separable(p, loc, X, wl.weight, T)
    model = O.degrid_separable(p, loc, _round_fp16(X.real) + 1j * _round_fp16(X.imag),
                               wl.weight, _round_fp16(T.real) + 1j * _round_fp16(T.imag))
    e_model = rel_l2(model, want)
    assert e_model > 1e-2  # the ill-conditioned regime
    _, _, ctx, taps, d = _grid(torch, S, wl, S.FORM_TC_FP16)
    out = torch.empty(wl.nvis, dtype=torch.complex64, device="cuda")
    S.sepw_degrid(ctx, taps, d["u"], d["v"], d["w"],
                  torch.from_numpy(X.astype(np.complex64)).cuda(), d["weight"], out)
    e_gpu = rel_l2(out.cpu().numpy(), want)
    assert 0.9 * e_model <= e_gpu <= 1.1 * e_model


@pytest.mark.parametrize("prec", ["fp16", "fp16x2", "bf16x2"])
def test_tc_degrid_heavy_tile(env, prec):
    """50,000 visibilities at one position: many stages and items on one
    window, in both buffers of each kind.  Each prediction is a short sum (no
    cancellation over many visibilities, unlike gridding), so the bars are
    the form's."""
    torch, S = env
    n = 60000
    rng = np.random.default_rng(4)
    fov = math.radians(2.0)
    u = np.concatenate([np.full(50000, 2.2 / fov), rng.uniform(-6, 6, n - 50000) / fov])
    v = np.concatenate([np.full(50000, -3.9 / fov), rng.uniform(-6, 6, n - 50000) / fov])
    w = rng.uniform(-300, 300, n)
    vis = np.zeros(n, np.complex64)
    wt = rng.uniform(0.5, 1, n).astype(np.float32)
    wl = synth.Workload("heavy", 96, fov, 16, 16, 9, 300.0, u, v, w, vis, wt)
    p = O.params_from(wl.params())
    loc = O.locate(p, u, v, w)
    X = (rng.standard_normal((96, 96)) + 1j * rng.standard_normal((96, 96))).astype(np.complex64)
    want = O.degrid_separable(p, loc, X, wt, O.taps(p))
    _, _, ctx, taps, d = _grid(torch, S, wl, _form(S, prec))
    out = torch.empty(n, dtype=torch.complex64, device="cuda")
    S.sepw_degrid(ctx, taps, d["u"], d["v"], d["w"], torch.from_numpy(X).cuda(), d["weight"],
                  out)
    assert S.sepw_device_status(ctx) == S.OK
    assert rel_l2(out.cpu().numpy(), want) <= TOL[prec]


def test_tc_empty_and_all_dropped(env):
    torch, S = env
    wl = CASES["rand_S12"]()
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TC_BF16))
    taps = S.sepw_make_taps(ctx)
    N = wl.grid_size
    grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    e = torch.empty(0, dtype=torch.float64, device="cuda")
    S.sepw_grid(ctx, taps, e, e, e, torch.empty(0, dtype=torch.complex64, device="cuda"),
                None, grid)
    far = torch.full((50,), 1e12, dtype=torch.float64, device="cuda")
    S.sepw_grid(ctx, taps, far, far, far, torch.ones(50, dtype=torch.complex64,
                                                     device="cuda"), None, grid)
    assert float(grid.abs().sum()) == 0.0
    assert S.sepw_device_status(ctx) == S.OK


def test_tc_meerkat_subsample_errors(env):
    """1% seeded subsample of the 32,256,000-visibility workload on the full
    4096^2 grid: each tensor-core form against the FP64 oracle."""
    torch, S = env
    wl = synth.meerkat_like()
    sub = wl.subsample(wl.nvis // 100)
    want, _ = _oracle(sub)
    for prec in PRECS:
        got, *_ = _grid(torch, S, sub, _form(S, prec))
        err = rel_l2(got, want)
        assert err <= TOL[prec], (prec, err)


@pytest.mark.parametrize("prec", ["bf16", "fp16x2", "tf32"])
def test_tc_wait_timeout_reported_and_recovered(env, prec):
    """The timeout path of the bounded waits: with the MMA thread stalled by
    the test hook and a 2 ms limit, the launch ends by itself with
    SEPW_ETIMEOUT recorded (nothing is left waiting, tensor memory is
    released), and the next launch on the same context is correct."""
    torch, S = env
    wl = CASES["rand_S16"]()
    want, _ = _oracle(wl)
    _, _, ctx, taps, d = _grid(torch, S, wl, _form(S, prec))
    N = wl.grid_size
    S.sepw_set_wait_limit(ctx, 2_000_000)
    S.sepw_test_stall_mma(ctx, True)
    g = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], g)
    out = torch.zeros(wl.nvis, dtype=torch.complex64, device="cuda")
    S.sepw_degrid(ctx, taps, d["u"], d["v"], d["w"], g, d["weight"], out)
    assert S.sepw_device_status(ctx) == S.ETIMEOUT
    assert S.sepw_device_status(ctx) == S.OK  # read and reset
    S.sepw_test_stall_mma(ctx, False)
    S.sepw_set_wait_limit(ctx, 2_000_000_000)
    g.zero_()
    S.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], g)
    assert S.sepw_device_status(ctx) == S.OK
    assert rel_l2(g.cpu().numpy(), want) <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16", "bf16x2", "tf32"])
@pytest.mark.parametrize("chunk", [64, 544])
def test_tc_schedule_item_sizes(env, prec, chunk):
    """Smaller work items (ragged 32-visibility stages, more items per CTA and
    so both tensor-memory accumulators in turn) give the oracle's grid."""
    torch, S = env
    wl = synth.random_case(83, 30000, 256, 16, 16, 33, edge_fraction=0.1, radius_cells=40.0)
    want, _ = _oracle(wl)
    ctx = S.sepw_create(S.make_params(**wl.params(), form=_form(S, prec)))
    S.sepw_set_schedule(ctx, chunk, 0)
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    N = wl.grid_size
    g = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], g)
    assert S.sepw_device_status(ctx) == S.OK
    assert rel_l2(g.cpu().numpy(), want) <= TOL[prec]


@pytest.mark.parametrize("support", [2, 4, 6, 10, 14])
@pytest.mark.parametrize("prec", PRECS)
def test_tc_other_supports(env, support, prec):
    """Supports whose taps do not fill the 16-tap table rows (zero padding,
    shifts of every residue, the largest tile T = 33 - S rounded to even):
    gridding and degridding against the oracle at the form's bar."""
    torch, S = env
    wl = synth.random_case(40 + support, 4000, 128, support, 8, 9, edge_fraction=0.1)
    p = O.params_from(wl.params())
    want, loc = _oracle(wl)
    got, _, ctx, taps, d = _grid(torch, S, wl, _form(S, prec))
    assert rel_l2(got, want) <= TOL[prec], (support, prec)
    N = wl.grid_size
    rng = np.random.default_rng(support)
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    want_p = O.degrid_separable(p, loc, X, wl.weight, O.taps(p))
    out = torch.zeros(wl.nvis, dtype=torch.complex64, device="cuda")
    S.sepw_degrid(ctx, taps, d["u"], d["v"], d["w"], torch.from_numpy(X).cuda(), d["weight"], out)
    assert S.sepw_device_status(ctx) == S.OK
    assert rel_l2(out.cpu().numpy(), want_p) <= TOL[prec], (support, prec)
