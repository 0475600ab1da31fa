"""Pins of the oracle's image-plane faceting (Sec. 4.1, Eq. gt-facet):
the centre facet reduces to the separable screen without its quartic term,
the full-support facet pipeline equals its direct sum, the facet screens are
the second-order Taylor expansion of h about the facet centre (the residual is
the dropped cross term -n0^-3 l0 m0 l m), and that residual scales with the
square of the facet width."""
import math

import numpy as np

import oracle as O


def test_centre_facet_is_separable_screen_without_quartic_term():
    p = O.Params(64, math.radians(6.0), 8, 8, 5, 500.0)
    Tu, Tv = O.taps_facet(p, 0.0, 0.0)
    T0 = O.taps(O.Params(64, math.radians(6.0), 8, 8, 5, 500.0, gamma=0.0))
    assert np.max(np.abs(Tu - T0)) < 1e-15 and np.max(np.abs(Tv - T0)) < 1e-15
    al, am = O.facet_coeffs(0.0, 0.0)
    assert al == am == -0.5


def test_facet_tables_differ_between_l_and_m():
    p = O.Params(64, math.radians(6.0), 8, 8, 5, 500.0)
    Tu, Tv = O.taps_facet(p, 0.2, -0.05)
    al, am = O.facet_coeffs(0.2, -0.05)
    n0 = math.sqrt(1 - 0.04 - 0.0025)
    assert abs(al + 0.5 * (1 / n0 + 0.04 / n0 ** 3)) < 1e-15
    assert abs(am + 0.5 * (1 / n0 + 0.0025 / n0 ** 3)) < 1e-15
    assert np.max(np.abs(Tu - Tv)) > 1e-3 * np.max(np.abs(Tu))
    # plane 0 (w = 0) has no screen: both tables equal the w = 0 taps
    assert np.max(np.abs(Tu[0] - O.taps(p)[0])) < 1e-15


def test_full_support_facet_pipeline_equals_direct_sum():
    """Full support (S = N, periodic), shifted positions on the oversampled
    grid, w on plane values >= 0: the facet image equals the direct sum."""
    N, OS, P, w_max = 32, 4, 5, 256.0
    p = O.Params(N, math.radians(8.0), N, OS, P, w_max, kb_beta=3.0)
    l0, m0 = 0.15, -0.1
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0)
    rng = np.random.default_rng(41)
    n = 12
    w = O.plane_w(P, w_max)[rng.integers(0, P, n)]
    xc = rng.integers(-N // 3, N // 3, n) + rng.integers(0, OS, n) / OS
    yc = rng.integers(-N // 3, N // 3, n) + rng.integers(0, OS, n) / OS
    # choose u, v so that the shifted u', v' sit on the oversampled grid
    u = xc / p.fov + w * l0 / n0
    v = yc / p.fov + w * m0 / n0
    up, vp, _ = O.facet_shift(u, v, w, np.ones(n), l0, m0)
    assert np.max(np.abs(up * p.fov - xc)) < 1e-9
    vis = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    wt = rng.uniform(0.5, 1, n)
    got = O.facet_image(p, l0, m0, u, v, w, vis, wt, wrap=True)
    want = O.dirty_direct_facet(p, l0, m0, u, v, w, vis, wt)
    assert np.max(np.abs(got - want)) < 1e-8 * np.max(np.abs(want))


def _facet_phase_residual(l0, m0, l, m):
    """h(l0 + l, m0 + m) - h(l0, m0) minus its facet approximation (the
    linear term and the two quadratic terms of Eq. gt-facet)."""
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0)
    al, am = O.facet_coeffs(l0, m0)
    h = np.sqrt(1 - (l0 + l) ** 2 - (m0 + m) ** 2)
    return (h - n0) - (-(l0 * l + m0 * m) / n0 + al * l * l + am * m * m)


def test_facet_screens_are_second_order_taylor_with_cross_term_dropped():
    l0, m0 = 0.2, 0.1
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0)
    for s in (1e-3, 2e-3):
        l = m = s
        res = _facet_phase_residual(l0, m0, l, m)
        cross = -l0 * m0 * l * m / n0 ** 3
        assert abs(res / cross - 1) < 20 * s  # remainder O(|l|^3)
    # with l0 m0 = 0 the cross term vanishes and the residual is third order
    r1 = _facet_phase_residual(0.2, 0.0, 1e-3, 1e-3)
    r2 = _facet_phase_residual(0.2, 0.0, 2e-3, 2e-3)
    assert abs(r2 / r1 - 8) < 0.05


def test_facet_error_scales_with_square_of_facet_width():
    """Sec. 4.1: the phase error over a facet now scales with the square of
    the facet width (the cross term), not the fourth power."""
    l0, m0 = 0.3, 0.3

    def max_err(width):
        x = np.linspace(-width / 2, width / 2, 41)
        L, M = np.meshgrid(x, x)
        return np.max(np.abs(_facet_phase_residual(l0, m0, L, M)))

    r = max_err(0.01) / max_err(0.005)
    assert 3.8 < r < 4.3
