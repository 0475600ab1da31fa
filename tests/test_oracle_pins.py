"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an
invariant, a value printed in the paper, a special case that reduces to a
textbook formula, or brute force with exact rational arithmetic.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _case(N=32, S=32, OS=4, P=5, fov=math.radians(8.0), w_max=300.0, beta=3.0,
          n=16, seed=1, neg=True, gamma=5.0 / 24.0, integer_pos=False):
    """Visibilities on the oversampled grid with w on plane values, for the
    full-support (S = N, periodic) pins.  A small taper beta keeps 1/c1 at
    the image edge moderate so that rounding is not amplified."""
    p = O.Params(N, fov, S, OS, P, w_max, gamma=gamma, kb_beta=beta)
    rng = np.random.default_rng(seed)
    fx = 0 if integer_pos else rng.integers(0, OS, n) / OS
    fy = 0 if integer_pos else rng.integers(0, OS, n) / OS
    xc = rng.integers(-N // 3, N // 3, n) + fx
    yc = rng.integers(-N // 3, N // 3, n) + fy
    u, v = xc / fov, yc / fov
    pl = rng.integers(0, P, n)
    sgn = np.where(rng.random(n) < 0.5, -1.0, 1.0) if neg else np.ones(n)
    w = O.plane_w(P, w_max)[pl] * sgn
    vis = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    wt = rng.uniform(0.5, 1.0, n)
    return p, u, v, w, vis, wt


# --------------------------------------------------------------------------
# taper and taps
# --------------------------------------------------------------------------


@pytest.mark.parametrize("S,beta", [(8, 18.72), (16, 37.44), (12, 28.08)])
def test_taper_is_transform_of_kb_window(S, beta):
    """c1 is the continuous Fourier transform of the KB window, normalised to
    c1(0) = 1: compare with numerical quadrature of I0(beta sqrt(1-(2x/S)^2))."""
    from scipy import integrate
    norm = S * math.sinh(beta) / beta
    for nu in [0.0, 0.05, 0.13, 0.31, 0.5, 0.9]:
        f = lambda x: O.kb_kernel(np.array([x]), S, beta)[0] * math.cos(2 * math.pi * x * nu)  # noqa: E731
        val, _ = integrate.quad(f, -S / 2, S / 2, limit=400, epsabs=0, epsrel=1e-12)
        got = O.kb_taper(np.array([nu]), S, beta)[0] * norm
        assert abs(got - val) <= 1e-9 * abs(O.kb_kernel(np.array([0.0]), S, beta)[0])


def test_taps_w0_imaginary_part_closed_form():
    """At w = 0 the taps are the DFT of the real, even taper over pixels
    a = 0..N-1; all terms pair off except the Nyquist pixel nu = -1/2, so
    Im F1_0(d) = c1(1/2) sin(pi d) / N exactly."""
    p = O.Params(64, math.radians(2.0), 8, 8, 3, 1000.0)
    T0 = O.taps(p)[0]
    d = O.tap_offsets(p.S, p.OS)
    c_nyq = O.kb_taper(np.array([0.5]), p.S, p.kb_beta)[0]
    want = c_nyq * np.sin(np.pi * d) / p.N
    assert np.max(np.abs(T0.imag - want)) < 1e-16 + 1e-13 * c_nyq


def test_taps_negative_w_is_conjugate_up_to_nyquist_term():
    """F1_{-w} = conj(F1_w) for the continuous transform (taper and screen are
    even); with the N-pixel DFT the only unpaired term is nu = -1/2, giving
    F1_{-w}(d) - conj F1_w(d) = (2i/N) c1(1/2) g1_{-w}(l_0) sin(pi d)."""
    pp = O.Params(64, math.radians(4.0), 16, 8, 4, 1500.0)
    pm = O.Params(64, math.radians(4.0), 16, 8, 4, -1500.0)
    Tp, Tm = O.taps(pp), O.taps(pm)
    d = O.tap_offsets(16, 8)
    c_nyq = O.kb_taper(np.array([0.5]), 16, pp.kb_beta)[0]
    l0 = O.pixel_l(64, pp.fov)[0]
    for k, wv in enumerate(O.plane_w(4, -1500.0)):
        want = 2j / 64 * c_nyq * O.g1(wv, l0, pp.gamma) * np.sin(np.pi * d)
        assert np.max(np.abs(Tm[k] - np.conj(Tp[k]) - want)) < 1e-15


@pytest.mark.parametrize("S,OS,N", [(8, 8, 256), (16, 16, 512)])
def test_taps_w0_match_kb_samples_within_tail_bound(S, OS, N):
    """At w = 0 the taps are the band-limited KB window: F1_0(d) equals
    C(d) beta / (S sinh beta) up to the taper's tail beyond |nu| = 1/2 and the
    end correction of the N-point sum (each bounded by the taper there)."""
    from scipy import integrate
    beta = 2.34 * S
    p = O.Params(N, math.radians(2.0), S, OS, 2, 100.0, kb_beta=beta)
    T0 = O.taps(p)[0]
    d = O.tap_offsets(S, OS)
    want = O.kb_kernel(d, S, beta) * beta / (S * math.sinh(beta))
    tail, _ = integrate.quad(lambda x: abs(O.kb_taper(np.array([x]), S, beta)[0]),
                             0.5, 40.0, limit=2000)
    c_nyq = O.kb_taper(np.array([0.5]), S, beta)[0]
    bound = 2 * tail + 2 * c_nyq / N + 1e-15
    err = np.max(np.abs(T0 - want))
    assert err <= bound
    # the bound is far below the peak, so a wrong scale or offset would fail
    assert bound < 5e-3 * np.max(np.abs(want))


def test_separable_table_is_outer_product_of_taps():
    """Eq. gt / Sec. 5: the 2-D kernel built from g~ = g1(l) g1(m) is the outer
    product F1_w(u) F1_w(v) of the 1-D taps."""
    p = O.Params(48, math.radians(6.0), 8, 4, 3, 800.0)
    T = O.taps(p)
    K = O.exact_table(p, screen="separable")
    outer = T[:, :, None, :, None] * T[:, None, :, None, :]  # [p][ov][ou][k][j]
    assert np.max(np.abs(K - outer)) < 1e-14 * np.max(np.abs(outer))


def test_w0_exact_kernel_equals_separable():
    """w = 0: g = g~ = 1, so the exact kernel is the separable one and the
    two gridders agree (W-projection reduces to plain gridding)."""
    p = O.Params(48, math.radians(6.0), 8, 4, 1, 800.0)
    T = O.taps(p)
    K = O.exact_table(p, screen="exact")
    outer = T[:, :, None, :, None] * T[:, None, :, None, :]
    assert np.max(np.abs(K - outer)) < 1e-14 * np.max(np.abs(outer))
    rng = np.random.default_rng(5)
    n = 300
    u = rng.uniform(-15, 15, n) / p.fov
    v = rng.uniform(-15, 15, n) / p.fov
    w = np.zeros(n)
    vis = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    loc = O.locate(p, u, v, w)
    g1_ = O.grid_separable(p, loc, vis, None, T)
    g2_ = O.grid_exact2d(p, loc, vis, None, K)
    assert np.max(np.abs(g1_ - g2_)) < 1e-13 * np.max(np.abs(g1_))


# --------------------------------------------------------------------------
# full pipeline against the direct sums (Eq. dirty, prediction integral)
# --------------------------------------------------------------------------


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_separable_pipeline_reproduces_direct_sum_w_nonneg():
    """Full support (S = N, periodic), visibilities on the oversampled grid,
    w on plane values >= 0: gridding + unnormalised inverse DFT + grid
    correction equals Eq. dirty with the separable screen g~, to round-off."""
    p, u, v, w, vis, wt = _case(neg=False)
    loc = O.locate(p, u, v, w, wrap=True)
    assert loc["keep"].all()
    g = O.grid_separable(p, loc, vis, wt, O.taps(p), wrap=True)
    img = O.grid_to_image_direct(p, g)
    d = O.dirty_direct(p.N, p.fov, u, v, w, vis, wt, screen="separable", gamma=p.gamma)
    assert _rel(img, d) < 1e-10


def test_separable_pipeline_negative_w_exact_off_nyquist():
    """With w < 0 (conjugate kernel) the identity still holds at every pixel
    except the Nyquist row and column (nu = -1/2), where it holds only for
    integer cell positions (the unpaired DFT term)."""
    p, u, v, w, vis, wt = _case(neg=True, seed=2)
    loc = O.locate(p, u, v, w, wrap=True)
    g = O.grid_separable(p, loc, vis, wt, O.taps(p), wrap=True)
    img = O.grid_to_image_direct(p, g)
    d = O.dirty_direct(p.N, p.fov, u, v, w, vis, wt, screen="separable", gamma=p.gamma)
    scale = np.max(np.abs(d))
    assert np.max(np.abs(img - d)[1:, 1:]) / scale < 1e-10
    p, u, v, w, vis, wt = _case(neg=True, seed=3, integer_pos=True)
    loc = O.locate(p, u, v, w, wrap=True)
    g = O.grid_separable(p, loc, vis, wt, O.taps(p), wrap=True)
    img = O.grid_to_image_direct(p, g)
    d = O.dirty_direct(p.N, p.fov, u, v, w, vis, wt, screen="separable", gamma=p.gamma)
    assert _rel(img, d) < 1e-10


def test_exact_pipeline_reproduces_direct_sum():
    """The exact 2-D kernel gridder reproduces Eq. dirty with the true screen
    g_w = exp(2 pi i w (n-1)) (W projection, Eq. wprojection)."""
    p, u, v, w, vis, wt = _case(neg=False, seed=4)
    loc = O.locate(p, u, v, w, wrap=True)
    g = O.grid_exact2d(p, loc, vis, wt, O.exact_table(p), wrap=True)
    img = O.grid_to_image_direct(p, g)
    d = O.dirty_direct(p.N, p.fov, u, v, w, vis, wt, screen="exact")
    assert _rel(img, d) < 1e-10


def test_prediction_pipeline_reproduces_prediction_integral():
    """IMAGE -> GRID then separable degridding (full support) equals the
    prediction sum with the separable screen, for w >= 0."""
    p, u, v, w, vis, wt = _case(neg=False, seed=6, n=10)
    rng = np.random.default_rng(7)
    img = rng.standard_normal((p.N, p.N)) + 1j * rng.standard_normal((p.N, p.N))
    grid = O.image_to_grid_direct(p, img)
    loc = O.locate(p, u, v, w, wrap=True)
    got = O.degrid_separable(p, loc, grid, None, O.taps(p), wrap=True)
    want = O.predict_direct(p.N, p.fov, img, u, v, w, screen="separable", gamma=p.gamma)
    assert _rel(got, want) < 1e-10


def test_dirty_direct_w0_is_plain_fourier_sum():
    """Textbook special case: at w = 0 the direct sum is n times the 2-D
    Fourier series sum_i V_i exp(2 pi i (u l + v m)), checked by brute force."""
    rng = np.random.default_rng(8)
    N, fov = 8, 0.2
    u = rng.uniform(-20, 20, 5)
    v = rng.uniform(-20, 20, 5)
    vis = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    d = O.dirty_direct(N, fov, u, v, np.zeros(5), vis)
    for b in range(N):
        for a in range(N):
            l = (a - N // 2) * fov / N
            m = (b - N // 2) * fov / N
            s = sum(vis[i] * complex(math.cos(2 * math.pi * (u[i] * l + v[i] * m)),
                                     math.sin(2 * math.pi * (u[i] * l + v[i] * m)))
                    for i in range(5))
            assert abs(d[b, a] - math.sqrt(1 - l * l - m * m) * s) < 1e-12


# --------------------------------------------------------------------------
# the approximation's error (Sec. 3)
# --------------------------------------------------------------------------


def _pipeline_eps(fov_deg, gamma, N=64, w=1000.0):
    """Phase error factor eps(l, m) measured through the pipeline: one
    visibility at the phase centre with w on a plane, gridded with the
    separable taps and with the exact 2-D kernel (full support); the image
    ratio is exp(2 pi i w eps)."""
    fov = math.radians(fov_deg)
    p = O.Params(N, fov, N, 1, 2, w, gamma=gamma, kb_beta=3.0)
    u = v = np.zeros(1)
    ww = np.array([w])
    vis = np.ones(1, complex)
    loc = O.locate(p, u, v, ww, wrap=True)
    gs = O.grid_separable(p, loc, vis, None, O.taps(p), wrap=True)
    ge = O.grid_exact2d(p, loc, vis, None, O.exact_table(p), wrap=True)
    ratio = O.grid_to_image_direct(p, gs) / O.grid_to_image_direct(p, ge)
    eps = np.angle(ratio) / (2 * np.pi * w)
    l = O.pixel_l(N, fov)
    L, M = np.meshgrid(l, l)
    return eps, L, M


def test_pipeline_phase_error_matches_eps_formula():
    """The image-plane phase of separable vs exact W projection is
    2 pi w eps(l, m) with eps = -(l^2/2 + g l^4 + m^2/2 + g m^4) - (n - 1)."""
    eps, L, M = _pipeline_eps(8.0, 5.0 / 24.0)
    want = O.eps_exact(L, M, 5.0 / 24.0)
    assert np.max(np.abs(eps - want)) < 1e-12


def test_fourth_power_law_and_minimax_gamma():
    """Sec. 3: with gamma = 5/24 the maximum |eps| over a square image is
    m_max^4 / 12 (m_max = fov / 2) to leading order, and log max|eps| grows
    with slope 4 in log fov."""
    gold = json.load(open(GOLDEN))
    g = gold["minimax_gamma"]["gamma_minimax"]
    ratio = gold["minimax_gamma"]["max_eps_over_mmax4"]
    fovs = np.array([1.0, 2.0, 4.0, 8.0])
    mx = []
    for f in fovs:
        eps, L, M = _pipeline_eps(f, g)
        m_max = math.radians(f) / 2
        mx.append(np.max(np.abs(eps)))
        # O(l^6) corrections are relatively ~ m_max^2
        assert abs(mx[-1] / m_max ** 4 - ratio) < 0.6 * m_max ** 2 + 1e-6
    slope = np.polyfit(np.log(np.radians(fovs)), np.log(mx), 1)[0]
    assert abs(slope - gold["separable_error_order"]["exponent"]) < 0.05


def test_gamma_one_eighth_exact_on_axes():
    """Sec. 3: gamma = 1/8 favours the axes: there eps is O(l^6) (l^6/16)."""
    eps, L, M = _pipeline_eps(16.0, 0.125)
    N = eps.shape[0]
    axis = np.concatenate([eps[N // 2, :], eps[:, N // 2]])
    lax = np.concatenate([L[N // 2, :], M[:, N // 2]])
    assert np.all(np.abs(axis) <= 1.05 * lax ** 6 / 16 + 1e-13)
    assert np.max(np.abs(eps)) > 100 * np.max(np.abs(axis))


def test_leading_eps_minimax_value():
    """Sec. 3: along the edge m = m_max the leading-order eps with
    gamma = 5/24 has maximum magnitude m_max^4 / 12, attained at l = 0 and
    l = m_max, and any other gamma does worse."""
    m = 0.03
    l = np.linspace(-m, m, 20001)
    best = np.max(np.abs(O.eps_leading(l, m, 5.0 / 24.0)))
    assert abs(best - m ** 4 / 12) < 1e-6 * m ** 4
    for gam in [0.18, 0.2, 0.22, 0.25, 0.125]:
        assert np.max(np.abs(O.eps_leading(l, m, gam))) >= best * (1 - 1e-9)


def test_errscale_worked_examples():
    """Sec. 3 worked examples of Eq. errscale: MeerKAT ~0.0018 Q^4 and
    SKA1-MID 0.39 Q^4 (printed to two significant figures)."""
    gold = json.load(open(GOLDEN))
    for key in ("errscale_meerkat", "errscale_ska1_mid"):
        e = gold[key]
        val = O.errscale(1.0, e["lambda_m"], e["D_m"], e["B_m"],
                         math.radians(e["elevation_deg"]))
        assert float(f"{val:.{e['printed_sig_figs']}g}") == e["printed"]


def test_wstack_ska1_mid_eps_bound():
    """Sec. 4.3: for a 10 degree field of view |eps| < 1e-5 everywhere."""
    gold = json.load(open(GOLDEN))["wstack_ska1_mid_10deg"]
    half = math.radians(gold["fov_deg"]) / 2
    l = np.linspace(-half, half, 801)
    L, M = np.meshgrid(l, l)
    assert np.max(np.abs(O.eps_exact(L, M, 5.0 / 24.0))) < gold["eps_bound"]


def test_amplitude_loss_formula():
    """Eq. amplitude-loss: <1 - cos(2 pi dw eps)> ~ 2/3 pi^2 eps^2 w_max^2 for
    dw uniform in [-w_max, w_max] (small phase)."""
    eps, w_max = 1e-6, 2000.0
    dw = np.linspace(-w_max, w_max, 200001)
    mean = np.mean(1 - np.cos(2 * np.pi * dw * eps))
    assert abs(mean - O.amplitude_loss(eps, w_max)) < 1e-3 * mean


def test_appendix_root_solves_lprime():
    """Appendix A: the smaller root y of the quadratic gives dl = y d with
    l' = l + dl satisfying Eq. lprime; y1 = (1 + l.d/n) eps approximates it."""
    l = np.array([0.02, -0.015])
    d = np.array([1.5, 2.0])
    eps = 3e-8
    y = O.delta_l_roots(l, d, eps)
    lp = l + y * d
    n = math.sqrt(1 - l @ l)
    lhs = lp + (math.sqrt(1 - lp @ lp) - 1) * d
    rhs = l + (n - 1 + eps) * d
    assert np.max(np.abs(lhs - rhs)) < 1e-15
    assert abs(O.delta_l_y1(l, d, eps) - y) < 1e-3 * abs(y)


def test_w_support_formula_limits():
    """Sec. 2 support formula: at w -> 0 it vanishes; for large w it tends to
    the geometric term w fov^2."""
    fov = math.radians(2.0)
    assert O.w_support(0.0, fov, 0.01) == 0.0
    w = 1e13
    assert abs(O.w_support(w, fov, 0.01) / (w * fov * fov) - 1) < 1e-3


def test_w_support_formula_interior():
    """Sec. 2 support formula where both of its terms matter.

    Hand-evaluated at w = 1000, fov = 0.02, eta = 0.01:
      (w fov / 2)^2 = 10^2 = 100;
      w^(3/2) fov / (2 pi eta) = 31622.7766 * 0.02 / 0.0628318531 = 10065.842;
      2 fov sqrt(100 + 10065.842) = 0.04 * 100.82580 = 4.033032.
    And at the crossover w* = (2 / (pi eta fov))^2, where the two terms are
    equal, the support is sqrt(2) w* fov^2 (each term alone gives w* fov^2)."""
    assert abs(O.w_support(1000.0, 0.02, 0.01) - 4.033032) < 2e-6
    fov, eta = 0.02, 0.01
    ws = (2.0 / (math.pi * eta * fov)) ** 2
    assert abs(O.w_support(ws, fov, eta) / (math.sqrt(2.0) * ws * fov * fov) - 1) < 1e-12
    # below the crossover the w^(3/2) term dominates: support ~ w^(3/4)
    r = O.w_support(ws * 1e-12 * 16, fov, eta) / O.w_support(ws * 1e-12, fov, eta)
    assert abs(r - 16 ** 0.75) < 1e-4


def test_n_wplanes_needed():
    """Sec. 2 number of w planes, pi w_max fov^2 / sqrt(2 dA).

    Hand-evaluated at w_max = 2e5, fov = 0.05, dA = 0.01:
      pi * 2e5 * 0.0025 = 1570.7963;  sqrt(0.02) = 0.14142136;
      1570.7963 / 0.14142136 = 11107.207.
    The paper says the count easily reaches 10^4 at low elevation with
    dA = 0.01: the SKA1-MID example of Sec. 3 (15 degree elevation, field
    lambda / D, w_max = B cos(a) / lambda) gives about 1.2e4."""
    assert abs(O.n_wplanes_needed(2e5, 0.05, 0.01) - 11107.207) < 2e-3
    # scaling: linear in w_max, quadratic in fov, inverse square root in dA
    base = O.n_wplanes_needed(1e4, 0.03, 0.02)
    assert abs(O.n_wplanes_needed(2e4, 0.03, 0.02) / base - 2) < 1e-12
    assert abs(O.n_wplanes_needed(1e4, 0.06, 0.02) / base - 4) < 1e-12
    assert abs(O.n_wplanes_needed(1e4, 0.03, 0.005) / base - 2) < 1e-12
    g = json.load(open(GOLDEN))["wplanes_low_elevation"]
    ska = json.load(open(GOLDEN))[g["telescope"]]
    lam, D, B, a = ska["lambda_m"], ska["D_m"], ska["B_m"], math.radians(ska["elevation_deg"])
    P = O.n_wplanes_needed(B * math.cos(a) / lam, lam / D, g["dA"])
    assert g["printed_order"] <= P < 10 * g["printed_order"]


# --------------------------------------------------------------------------
# locating visibilities: brute-force rule checks with exact rationals
# --------------------------------------------------------------------------


def test_locate_rounding_invariants_exact_rationals():
    """0 <= o < OS and the oversampled position c + o/OS is the nearest
    multiple of 1/OS to x = u fov + N/2 (computed exactly from the doubles,
    up to the two roundings of the float evaluation)."""
    p = O.Params(256, math.radians(2.0), 8, 8, 32, 2000.0)
    rng = np.random.default_rng(11)
    u = rng.uniform(-100, 100, 400) / p.fov
    loc = O.locate(p, u, np.zeros_like(u), np.zeros_like(u))
    for i in range(len(u)):
        x = Fraction(float(u[i])) * Fraction(p.fov) + 128
        q = Fraction(int(loc["cu"][i])) + Fraction(int(loc["ou"][i]), 8)
        assert 0 <= loc["ou"][i] < 8
        assert abs(q - x) <= Fraction(1, 16) + Fraction(1, 10 ** 9)


def test_locate_ties_round_up_and_footprint_edges():
    """Exact ties x*OS + 1/2 = integer go to +inf; the first and last
    footprint positions inside [0, N) are kept, one cell further is dropped."""
    N, S, OS = 64, 8, 4
    fov = 2.0 ** -6  # makes u * fov exact
    p = O.Params(N, fov, S, OS, 3, 100.0)
    xs, want_c, want_o, want_keep = [], [], [], []
    for c, o in [(10, 1), (20, 3), (31, 0)]:
        xs.append(c + (o + 0.5) / OS)       # tie -> rounds up
        t = c * OS + o + 1
        want_c.append(t // OS)
        want_o.append(t % OS)
        want_keep.append(True)
    lo = S // 2 - 1           # first c whose footprint starts at cell 0
    hi = N - 1 - S // 2       # last c whose footprint ends at cell N-1
    for c, keep in [(lo, True), (lo - 1, False), (hi, True), (hi + 1, False)]:
        xs.append(float(c))
        want_c.append(c)
        want_o.append(0)
        want_keep.append(keep)
    u = (np.array(xs) - N / 2) / fov
    loc = O.locate(p, u, np.zeros_like(u) + 0.0, np.zeros_like(u))
    for i in range(len(xs)):
        assert bool(loc["keep"][i]) == want_keep[i]
        if want_keep[i]:
            assert (loc["cu"][i], loc["ou"][i]) == (want_c[i], want_o[i])


def test_locate_planes_conj_and_nonfinite():
    """plane = round-half-up(|w| (P-1)/w_max); beyond plane P-1 (|w| >= w_max
    (1 + 1/(2(P-1)))) is dropped; w < 0 sets conj, -0.0 does not; NaN and
    inf coordinates are dropped."""
    P, w_max = 5, 400.0
    p = O.Params(64, 2.0 ** -6, 8, 4, P, w_max)
    w = np.array([0.0, -0.0, 50.0, 49.9, -150.0, 400.0, -449.0, 450.0, 451.0,
                  np.nan, np.inf, 10.0, 10.0])
    u = np.zeros_like(w)
    v = np.zeros_like(w)
    u[11] = np.nan
    v[12] = -np.inf
    loc = O.locate(p, u, v, w)
    q = [Fraction(float(abs(x))) * Fraction(P - 1) / Fraction(w_max) if np.isfinite(x)
         else None for x in w]
    for i in range(9):
        want = math.floor(q[i] + Fraction(1, 2))
        assert bool(loc["keep"][i]) == (want <= P - 1)
        if want <= P - 1:
            assert loc["plane"][i] == want
    assert list(loc["conj"][:5]) == [False, False, False, False, True]
    assert not loc["keep"][9:].any()


# --------------------------------------------------------------------------
# adjointness and the image step
# --------------------------------------------------------------------------


def test_grid_degrid_adjoint():
    """<grid(V), X> = <V, degrid(X)> (degridding is the adjoint of gridding,
    including the weights), on a random case with dropped visibilities."""
    import synth
    wl = synth.random_case(3, 2000, 64, 8, 8, 9, w_max=300.0)
    p = O.params_from(wl.params())
    T = O.taps(p)
    loc = O.locate(p, wl.u, wl.v, wl.w)
    assert 0 < loc["keep"].sum() < len(wl.u)
    rng = np.random.default_rng(12)
    V = rng.standard_normal(wl.nvis) + 1j * rng.standard_normal(wl.nvis)
    X = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    G = O.grid_separable(p, loc, V, wl.weight, T)
    D = O.degrid_separable(p, loc, X, wl.weight, T)
    lhs = np.vdot(G, X)
    rhs = np.vdot(V, D)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_image_step_fft_equals_direct_dft():
    p = O.Params(32, math.radians(4.0), 8, 4, 3, 100.0)
    rng = np.random.default_rng(13)
    G = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    a, b = O.grid_to_image(p, G), O.grid_to_image_direct(p, G)
    assert _rel(a, b) < 1e-12
    a, b = O.image_to_grid(p, G), O.image_to_grid_direct(p, G)
    assert _rel(a, b) < 1e-12


def test_image_to_grid_is_scaled_adjoint_of_grid_to_image():
    """IMAGE -> GRID = F diag(1/(n c c)); GRID -> IMAGE = diag(n/(c c)) F^H, so
    <image_to_grid(I), G> = <I, grid_to_image(G) / n^2>."""
    p = O.Params(16, math.radians(30.0), 8, 4, 3, 100.0)
    rng = np.random.default_rng(14)
    I = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    G = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    l = O.pixel_l(16, p.fov)
    L, M = np.meshgrid(l, l)
    n2 = 1 - L * L - M * M
    lhs = np.vdot(O.image_to_grid_direct(p, I), G)
    rhs = np.vdot(I, O.grid_to_image_direct(p, G) / n2)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
