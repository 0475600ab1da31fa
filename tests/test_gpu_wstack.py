"""Hybrid W stacking (Sec. 4.3) through the C ABI against the FP64 oracle:
slice assignment bit-exact, dropped counts, slice grids, the dirty image and
the prediction, for the FP32 tiled form and the FP16 hi + lo tensor-core
form (both held to the FP32 bar, 1e-5)."""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
CENTRES = np.array([-2400.0, -1200.0, -500.0, -150.0, 0.0, 150.0, 500.0, 1200.0, 2400.0])
W_MAX = 600.0  # largest half-gap between neighbouring centres


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


def _case(seed=61, nvis=12000, N=256, S=8):
    """Disk of (u, v) with w spread over the slices; a few w on exact
    midpoints (ties), beyond the outer slices (dropped), non-finite, -0.0."""
    wl = synth.random_case(seed, nvis, N, S, 8, 17, w_max=W_MAX, edge_fraction=0.05)
    rng = np.random.default_rng(seed + 1)
    w = rng.uniform(-3000.0, 3000.0, nvis)
    mids = (CENTRES[1:] + CENTRES[:-1]) / 2
    w[:len(mids)] = mids
    w[len(mids):2 * len(mids)] = CENTRES[:len(mids)]
    w[20] = np.nan
    w[21] = np.inf
    w[22] = -0.0
    w[23] = 3100.0
    wl.w = w
    return wl


def _dev(torch, wl):
    return {k: torch.from_numpy(np.ascontiguousarray(getattr(wl, k))).cuda()
            for k in ("u", "v", "w", "vis", "weight")}


def _plan(torch, S, wl, form):
    ctx = S.sepw_create(S.make_params(**dict(wl.params(), w_max=W_MAX), form=form))
    taps = S.sepw_make_taps(ctx)
    d = _dev(torch, wl)
    sl = torch.empty(wl.nvis, dtype=torch.int32, device="cuda")
    S.sepw_wstack_plan(ctx, CENTRES, d["u"], d["v"], d["w"], slice_out=sl)
    return ctx, taps, d, sl


def _params(wl):
    return O.params_from(dict(wl.params(), w_max=W_MAX))


def test_wstack_slices_and_drops(env):
    torch, S = env
    wl = _case()
    ctx, taps, d, sl = _plan(torch, S, wl, S.FORM_TILED)
    want, wr = O.wstack_assign(wl.w, CENTRES)
    assert np.array_equal(sl.cpu().numpy(), want.astype(np.int32))
    p = _params(wl)
    loc = O.locate(p, wl.u, wl.v, wr)
    nd = S.sepw_plan_dropped(ctx)
    assert nd == int((~loc["keep"]).sum())
    assert nd >= 3  # nan, inf and the residual beyond w_max


@pytest.mark.parametrize("form", ["tiled", "tc_fp16x2", "tc_bf16x2"])
def test_wstack_slice_grids_and_image(env, form):
    torch, S = env
    wl = _case()
    f = {"tiled": S.FORM_TILED, "tc_fp16x2": S.FORM_TC_FP16X2,
         "tc_bf16x2": S.FORM_TC_BF16X2}[form]
    ctx, taps, d, _ = _plan(torch, S, wl, f)
    N, L = wl.grid_size, len(CENTRES)
    grids = torch.zeros((L, N, N), dtype=torch.complex64, device="cuda")
    S.sepw_grid_planned(ctx, taps, d["vis"], d["weight"], grids)
    p = _params(wl)
    want, _, _ = O.wstack_layer_grids(p, wl.u, wl.v, wl.w, wl.vis, wl.weight, CENTRES)
    assert rel_l2(grids.cpu().numpy(), want) <= TOL
    img = torch.empty((N, N), dtype=torch.complex64, device="cuda")
    S.sepw_wstack_image(ctx, grids, img)
    want_img = sum(O.grid_to_image(p, want[c]) * O.wstack_phase(p, wc)
                   for c, wc in enumerate(CENTRES))
    # The grid correction n / (c1 c1) reaches ~1e7 at the corners for S = 8
    # and amplifies the FP32 rounding of the grids there, while the signal is
    # tapered before it is corrected: compare every pixel with the correction
    # divided out (exact weights), so the grid's error bar carries over.
    nu = O.pixel_nu(N)
    c1 = O.kb_taper(nu, p.S, p.kb_beta)
    l = nu * p.fov
    L_, M_ = np.meshgrid(l, l)
    wgt = c1[None, :] * c1[:, None] / np.sqrt(1 - L_ * L_ - M_ * M_)
    assert rel_l2(img.cpu().numpy() * wgt, want_img * wgt) <= TOL


def test_wstack_prediction(env):
    torch, S = env
    wl = _case(seed=71, nvis=8000)
    ctx, taps, d, _ = _plan(torch, S, wl, S.FORM_TILED)
    N, L = wl.grid_size, len(CENTRES)
    rng = np.random.default_rng(72)
    model = np.zeros((N, N), np.complex64)
    inner = slice(N // 4, 3 * N // 4)
    model[inner, inner] = rng.standard_normal((N // 2, N // 2))
    grids = torch.empty((L, N, N), dtype=torch.complex64, device="cuda")
    S.sepw_wstack_model_grids(ctx, torch.from_numpy(model).cuda(), grids)
    out = torch.full((wl.nvis,), complex(5, 5), dtype=torch.complex64, device="cuda")
    S.sepw_degrid_planned(ctx, taps, grids, d["weight"], out)
    p = _params(wl)
    mg = O.wstack_model_grids(p, model, CENTRES)
    assert rel_l2(grids.cpu().numpy(), mg) <= TOL
    layer, wr = O.wstack_assign(wl.w, CENTRES)
    T = O.taps(p)
    want = np.zeros(wl.nvis, np.complex128)
    for c in range(L):
        sel = np.nonzero(layer == c)[0]
        if len(sel):
            loc = O.locate(p, wl.u[sel], wl.v[sel], wr[sel])
            want[sel] = O.degrid_separable(p, loc, mg[c], wl.weight[sel], T)
    got = out.cpu().numpy()
    assert rel_l2(got, want) <= TOL
    loc_all = O.locate(p, wl.u, wl.v, wr)
    assert np.all(got[~loc_all["keep"]] == 0)


def test_wstack_rejects(env):
    torch, S = env
    wl = _case(nvis=200)
    d = _dev(torch, wl)
    ctx = S.sepw_create(S.make_params(**dict(wl.params(), w_max=W_MAX), form=S.FORM_PLAIN))
    with pytest.raises(S.SepwError) as e:
        S.sepw_wstack_plan(ctx, CENTRES, d["u"], d["v"], d["w"])
    assert e.value.status == S.ENOTSUP
    ctx = S.sepw_create(S.make_params(**dict(wl.params(), w_max=W_MAX), form=S.FORM_TILED))
    for bad in ([0.0, 0.0], [1.0, 0.0], [0.0, np.nan], []):
        with pytest.raises(S.SepwError) as e:
            S.sepw_wstack_plan(ctx, bad, d["u"], d["v"], d["w"])
        assert e.value.status == S.EINVAL
