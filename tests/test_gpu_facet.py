"""Image-plane faceting (Sec. 4.1, Eq. gt-facet) through the C ABI against the
FP64 oracle: facet tap tables, the uv shift (bit-exact) and phase rotation,
gridding with separate u and v tables in every form, the facet image step and
prediction back to the original phase centre."""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

L0, M0 = 0.012, -0.007  # facet centre (direction cosines)


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
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(S_=8, seed=91, nvis=8000, N=128):
    return synth.random_case(seed, nvis, N, S_, 8, 9, w_max=400.0, radius_cells=40.0)


def _ctx(S, wl, form):
    ctx = S.sepw_create(S.make_params(**wl.params(), form=form))
    S.sepw_set_facet(ctx, L0, M0)
    return ctx


def test_facet_taps(env):
    torch, S = env
    wl = _case()
    ctx = _ctx(S, wl, S.FORM_TILED)
    p = O.params_from(wl.params())
    Tu, Tv = O.taps_facet(p, L0, M0)
    t64 = S.sepw_make_taps_f64(ctx).cpu().numpy()
    assert t64.shape == (2,) + Tu.shape
    assert np.max(np.abs(t64[0] - Tu)) < 1e-12 and np.max(np.abs(t64[1] - Tv)) < 1e-12
    t32 = S.sepw_make_taps(ctx).cpu().numpy()
    assert np.max(np.abs(t32 - t64)) <= 2 ** -24 * np.max(np.abs(t64)) * 1.01
    # facet mode off: one table of Eq. gt again
    S.sepw_set_facet(ctx, None)
    t = S.sepw_make_taps_f64(ctx).cpu().numpy()
    assert np.max(np.abs(t - O.taps(p))) < 1e-12


def test_facet_shift_bit_exact_uv(env):
    torch, S = env
    wl = _case()
    ctx = _ctx(S, wl, S.FORM_TILED)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis")}
    uo, vo = torch.empty_like(d["u"]), torch.empty_like(d["v"])
    vso = torch.empty_like(d["vis"])
    S.sepw_facet_shift(ctx, S.FACET_IN, d["u"], d["v"], d["w"], d["vis"], uo, vo, vso)
    up, vp, visp = O.facet_shift(wl.u, wl.v, wl.w, wl.vis, L0, M0)
    assert np.array_equal(uo.cpu().numpy(), up) and np.array_equal(vo.cpu().numpy(), vp)
    assert rel_l2(vso.cpu().numpy(), visp) < 1e-6
    back = torch.empty_like(vso)
    S.sepw_facet_shift(ctx, S.FACET_OUT, d["u"], d["v"], d["w"], vso, None, None, back)
    assert rel_l2(back.cpu().numpy(), wl.vis) < 1e-6


@pytest.mark.parametrize("S_,form", [(8, "tiled"), (10, "tiled"), (16, "tiled"),
                                     (8, "plain"), (16, "tc_fp16x2"), (16, "tc_bf16x2"),
                                     (16, "tc_bf16")])
def test_facet_grid_image_and_prediction(env, S_, form):
    """Gridding, image step and prediction with the facet tables (separate u-
    and v-tap tables, the v taps at an offset): the FP32 forms and the hi + lo
    tensor-core forms at 1e-5, the BF16 tensor-core form at its 1e-2."""
    torch, S = env
    wl = _case(S_=S_, seed=92 + S_)
    f = {"tiled": S.FORM_TILED, "plain": S.FORM_PLAIN, "tc_fp16x2": S.FORM_TC_FP16X2,
         "tc_bf16x2": S.FORM_TC_BF16X2, "tc_bf16": S.FORM_TC_BF16}[form]
    tol = 1e-2 if form == "tc_bf16" else 1e-5
    ctx = _ctx(S, wl, f)
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    uo, vo = torch.empty_like(d["u"]), torch.empty_like(d["v"])
    vso = torch.empty_like(d["vis"])
    S.sepw_facet_shift(ctx, S.FACET_IN, d["u"], d["v"], d["w"], d["vis"], uo, vo, vso)
    N = wl.grid_size
    grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S.sepw_grid(ctx, taps, uo, vo, d["w"], vso, d["weight"], grid)
    p = O.params_from(wl.params())
    up, vp, visp = O.facet_shift(wl.u, wl.v, wl.w, wl.vis, L0, M0)
    loc = O.locate(p, up, vp, wl.w)
    Tu, Tv = O.taps_facet(p, L0, M0)
    want = O.grid_separable(p, loc, visp, wl.weight, Tu, Tv=Tv)
    assert rel_l2(grid.cpu().numpy(), want) <= tol
    # image step with n at the facet's pixels; compare with the grid
    # correction divided out (it amplifies FP32 rounding at the facet edge)
    S.sepw_image(ctx, S.GRID_TO_IMAGE, grid)
    want_img = O.grid_to_image(p, want, L0, M0)
    nu = O.pixel_nu(N)
    c1 = O.kb_taper(nu, p.S, p.kb_beta)
    l = nu * p.fov
    n = np.sqrt(1 - (l[None, :] + L0) ** 2 - (l[:, None] + M0) ** 2)
    wgt = c1[None, :] * c1[:, None] / n
    assert rel_l2(grid.cpu().numpy() * wgt, want_img * wgt) <= tol
    # prediction: degrid a model grid with the facet tables, rotate back
    rng = np.random.default_rng(S_)
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    out = torch.empty_like(vso)
    S.sepw_degrid(ctx, taps, uo, vo, d["w"], torch.from_numpy(X).cuda(), d["weight"], out)
    S.sepw_facet_shift(ctx, S.FACET_OUT, d["u"], d["v"], d["w"], out, None, None, out)
    n0 = math.sqrt(1 - L0 * L0 - M0 * M0)
    ph = wl.u * L0 + wl.v * M0 + wl.w * (n0 - 1.0)
    wantv = O.degrid_separable(p, loc, X, wl.weight, Tu, Tv=Tv) * np.exp(-2j * np.pi * ph)
    assert rel_l2(out.cpu().numpy(), wantv) <= tol


def test_facet_rejects(env):
    torch, S = env
    wl = _case(nvis=100)
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TILED))
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w")}
    uo = torch.empty_like(d["u"])
    with pytest.raises(S.SepwError) as e:
        S.sepw_facet_shift(ctx, S.FACET_IN, d["u"], d["v"], d["w"], None, uo, uo.clone())
    assert e.value.status == S.ENOTSUP
    for bad in ((1.0, 0.1), (float("nan"), 0.0)):
        with pytest.raises(S.SepwError) as e:
            S.sepw_set_facet(ctx, *bad)
        assert e.value.status == S.EINVAL
