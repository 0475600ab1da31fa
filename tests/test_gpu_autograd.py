"""torch.autograd over the C ABI: Grid (backward = degridding) and Predict
(IMAGE_TO_GRID + degridding; backward = gridding + the adjoint image step),
against the FP64 oracle's analytic gradient and central finite differences."""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_07152_gb300 import build
    build.build()
    import paper_1511_07152_gb300.sepw as S
    from paper_1511_07152_gb300 import autograd as AG
    return torch, S, AG


def rel_l2(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _setup(torch, S, wl, form=1):
    ctx = S.sepw_create(S.make_params(**wl.params(), form=form))
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    S.sepw_plan(ctx, d["u"], d["v"], d["w"])
    return ctx, taps, d


def test_grid_backward_is_degridding(env):
    torch, S, AG = env
    wl = synth.random_case(41, 5000, 128, 8, 8, 9, w_max=300.0)
    ctx, taps, d = _setup(torch, S, wl)
    vis = d["vis"].clone().requires_grad_(True)
    G = AG.grid(vis, ctx, taps, d["weight"])
    rng = np.random.default_rng(2)
    X = torch.from_numpy((rng.standard_normal((128, 128)) +
                          1j * rng.standard_normal((128, 128))).astype(np.complex64)).cuda()
    # L = Re <X, G>  =>  dL/dvis* = A^H X / 2 in torch's convention: grad = A^H X
    L = (X.conj() * G).real.sum()
    L.backward()
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    want = O.degrid_separable(p, loc, X.cpu().numpy(), wl.weight, O.taps(p))
    assert rel_l2(vis.grad.cpu().numpy(), want) <= 1e-5


def _oracle_grad(wl, image, target):
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    T = O.taps(p)
    r = O.degrid_separable(p, loc, O.image_to_grid(p, image), None, T) - target
    G = O.grid_separable(p, loc, wl.weight.astype(np.float64) * r, None, T)
    l = O.pixel_l(p.N, p.fov)
    L, M = np.meshgrid(l, l)
    return 2 * np.real(O.grid_to_image(p, G) / (1 - L * L - M * M))


@pytest.mark.parametrize("form", [1, 3, 5])
def test_predict_gradient_matches_oracle(env, form):
    """Gradient of sum_i W_i |Predict(I)_i - V_i|^2 w.r.t. a real image."""
    torch, S, AG = env
    wl = synth.random_case(42, 6000, 128, 8, 8, 9, w_max=300.0, radius_cells=50.0)
    ctx, taps, d = _setup(torch, S, wl, form=form)
    rng = np.random.default_rng(3)
    image = rng.standard_normal((128, 128))
    if form in (3, 5):
        # FP16 degridding errs relative to the model grid, not to the
        # prediction: a white image divided by n c1^2 gives a grid 500 times
        # the prediction's rms (degridding cancels the edge-amplified part),
        # and 11-bit operands then cost 3% of the prediction (pinned in the
        # tensor-core tests).  The model here is tapered, x = n c1 c1 y, the
        # parameterisation of the major cycles, where the grid is 3 times the
        # prediction's rms.
        p = O.params_from(wl.params())
        c = O.kb_taper(O.pixel_nu(128), p.S, p.kb_beta)
        l = O.pixel_l(128, p.fov)
        image = image * np.sqrt(1.0 - l[None, :] ** 2 - l[:, None] ** 2) * np.outer(c, c)
    image = image.astype(np.float32)
    I = torch.from_numpy(image).cuda().requires_grad_(True)
    target = d["vis"]
    loss = AG.chi2(AG.predict(I, ctx, taps), target, d["weight"])
    loss.backward()
    want = _oracle_grad(wl, image.astype(np.float64), wl.vis.astype(np.complex128))
    got = I.grad.cpu().numpy()
    if form == 1:
        assert rel_l2(got, want) <= 1e-4
    elif form == 5:
        # BF16 hi + lo: grid and prediction errors ~4e-6, raised by the grid
        # correction's c1(0)^2 / c1(nu)^2 <= 7.8 inside |nu| < 1/4 (see
        # below): the FP32 bar holds there
        nu = O.pixel_nu(128)
        inner = np.ix_(np.abs(nu) < 0.25, np.abs(nu) < 0.25)
        assert rel_l2(got[inner], want[inner]) <= 1e-4
    else:
        # The tensor-core form grids the backward with FP16 operands (grid
        # error ~4e-4; the FP16 forward adds ~2e-4 on this model).  That rounding noise is white in the image domain,
        # while the gradient itself is tapered by c1^2 (it is gridded with
        # the taper), so the grid correction raises the relative error by
        # c1(0)^2 / c1(nu)^2: at most 7.8 inside |nu| < 1/4 for support 8,
        # hence the bar 7.8 x 4e-4 ~ 3e-3 there.
        nu = O.pixel_nu(128)
        inner = np.ix_(np.abs(nu) < 0.25, np.abs(nu) < 0.25)
        assert rel_l2(got[inner], want[inner]) <= 3e-3


def test_predict_finite_differences_literal(env):
    """Literal central differences, step 1e-3, on a well-conditioned case
    (model confined to |nu| < 1/4, where the grid correction 1/c1^2 stays
    below 8): the FP32 forward's rounding is small against the differences."""
    torch, S, AG = env
    wl = synth.random_case(43, 20000, 256, 8, 8, 9, w_max=300.0, radius_cells=100.0)
    ctx, taps, d = _setup(torch, S, wl)
    rng = np.random.default_rng(5)
    nu = O.pixel_nu(256)
    inner = np.abs(nu) < 0.25
    image = np.zeros((256, 256), np.float32)
    image[np.ix_(inner, inner)] = rng.standard_normal((inner.sum(), inner.sum()))
    I = torch.from_numpy(image).cuda()
    target = d["vis"]
    Ig = I.clone().requires_grad_(True)
    AG.chi2(AG.predict(Ig, ctx, taps), target, d["weight"]).backward()
    g = Ig.grad.cpu().numpy()
    h = 1e-3
    pix = rng.integers(80, 176, size=(32, 2))
    fd = []
    with torch.no_grad():
        for b, a in pix:
            e = torch.zeros_like(I)
            e[b, a] = h
            lp = AG.chi2(AG.predict(I + e, ctx, taps), target, d["weight"]).item()
            lm = AG.chi2(AG.predict(I - e, ctx, taps), target, d["weight"]).item()
            fd.append((lp - lm) / (2 * h))
    gp = g[pix[:, 0], pix[:, 1]]
    assert np.max(np.abs(np.array(fd) - gp)) <= 1e-2 * np.max(np.abs(gp))


def test_predict_finite_differences_point_source_model(env):
    """Workload 4: 2048^2 model of 500 point sources + N(0, 1e-4^2) noise,
    ~4M visibilities (support 16, oversampling 16, 64 planes), target =
    Predict(model) + N(0, 0.01^2); central differences on 64 seeded pixels.

    The loss L(I) = sum_i W_i |P(I)_i - V_i|^2 is quadratic in the image and P
    is linear, so the central difference with any step h is exactly
        (L(I + h e) - L(I - h e)) / (2h) = 2 Re <W r, P(e)>,  r = P(I) - V.
    The right-hand side is evaluated (P(e) is the forward of the single-pixel
    image e) rather than the left: the model's noise floor reaches the image
    edge, where the grid correction 1/c1^2 is ~1e8, so two FP32 predictions of
    the full image differ by rounding far more than by the step.  The check
    is then that the backward pass equals these differences to FP32 rounding
    (1e-4 of the largest derivative)."""
    torch, S, AG = env
    model, wl = synth.point_source_model()
    ctx, taps, d = _setup(torch, S, wl)
    I = torch.from_numpy(model).cuda()
    with torch.no_grad():
        clean = AG.predict(I, ctx, taps)
    rng = np.random.default_rng(151107152 * 10 + 40)
    noise = (0.01 * (rng.standard_normal(wl.nvis) + 1j * rng.standard_normal(wl.nvis))
             ).astype(np.complex64)
    target = clean + torch.from_numpy(noise).cuda()
    Ig = I.clone().requires_grad_(True)
    loss = AG.chi2(AG.predict(Ig, ctx, taps), target, d["weight"])
    loss.backward()
    grad = Ig.grad.cpu().numpy()
    N = wl.grid_size
    pix = rng.integers(N // 4, 3 * N // 4, size=(64, 2))
    wr = (d["weight"].to(torch.float64) * (clean.to(torch.complex128) -
                                           target.to(torch.complex128)))
    fd = []
    with torch.no_grad():
        for b, a in pix:
            e = torch.zeros_like(I)
            e[b, a] = 1.0
            pe = AG.predict(e, ctx, taps).to(torch.complex128)
            fd.append(float(2 * (wr.conj() * pe).real.sum()))
    fd = np.array(fd)
    g = grad[pix[:, 0], pix[:, 1]]
    assert np.max(np.abs(fd - g)) <= 1e-4 * np.max(np.abs(g))
