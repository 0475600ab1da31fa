"""Pins of the oracle's stored correction F_w - F~_w (Sec. 7): with the full
table the separable gridder plus the correction pass is the exact 2-D
W-projection gridder; the correction vanishes at w = 0; the correction's
degridder is its adjoint; and truncated or coarser tables still bring the
separable grid closer to the exact one."""
import math

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def case():
    p = O.Params(64, math.radians(6.0), 8, 8, 5, 800.0)
    rng = np.random.default_rng(1)
    n = 500
    u = rng.uniform(-20, 20, n) / p.fov
    v = rng.uniform(-20, 20, n) / p.fov
    w = rng.uniform(-800, 800, n)
    vis = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    wt = rng.uniform(0.5, 1, n)
    loc = O.locate(p, u, v, w)
    K = O.exact_table(p)
    T = O.taps(p)
    exact = O.grid_exact2d(p, loc, vis, wt, K)
    return p, loc, vis, wt, K, T, exact, rng


def test_full_correction_gives_exact_w_projection(case):
    p, loc, vis, wt, K, T, exact, _ = case
    assert np.any(loc["conj"] & loc["keep"]) and np.any(~loc["conj"] & loc["keep"])
    R = O.residual_table(p, K=K, T=T)
    g = O.grid_separable(p, loc, vis, wt, T)
    sep_err = np.max(np.abs(g - exact)) / np.max(np.abs(exact))
    O.grid_residual(p, loc, vis, wt, R, grid=g)
    assert np.max(np.abs(g - exact)) < 1e-13 * np.max(np.abs(exact))
    assert sep_err > 1e-6  # the correction is not trivially zero


def test_correction_vanishes_at_w0(case):
    p, _, _, _, K, T, _, _ = case
    R = O.residual_table(p, K=K, T=T)
    assert np.max(np.abs(R[0])) < 1e-14 * np.max(np.abs(K))
    assert np.max(np.abs(R[-1])) > 1e-6 * np.max(np.abs(K))


def test_correction_degrid_is_adjoint(case):
    p, loc, _, wt, K, T, _, rng = case
    R = O.residual_table(p, 4, 4, K=K, T=T)
    n = len(loc["keep"])
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = rng.standard_normal((p.N, p.N)) + 1j * rng.standard_normal((p.N, p.N))
    g = O.grid_residual(p, loc, x, wt, R)
    y = O.degrid_residual(p, loc, X, wt, R)
    lhs = np.vdot(X, g)
    rhs = np.vdot(y, x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("Sr,OSr,gain", [(8, 4, 3.0), (6, 8, 1.5), (4, 4, 1.1)])
def test_truncated_or_coarser_correction_still_helps(case, Sr, OSr, gain):
    p, loc, vis, wt, K, T, exact, _ = case
    gs = O.grid_separable(p, loc, vis, wt, T)
    e0 = np.linalg.norm(gs - exact)
    R = O.residual_table(p, Sr, OSr, K=K, T=T)
    O.grid_residual(p, loc, vis, wt, R, grid=gs)
    assert np.linalg.norm(gs - exact) * gain < e0


def test_residual_table_rejects_bad_sizes(case):
    p = case[0]
    for Sr, OSr in ((3, 8), (10, 8), (8, 3), (0, 8)):
        with pytest.raises(ValueError):
            O.residual_table(p, Sr, OSr)
