"""Pin of the oracle's gradient of the weighted chi-squared of prediction
(used as the reference for the autograd path): central finite differences in
FP64.  The loss is quadratic in the image, so central differences carry no
truncation error and match the analytic gradient to rounding."""
import math

import numpy as np

import oracle as O


def _predict(p, loc, T, image):
    return O.degrid_separable(p, loc, O.image_to_grid(p, image), None, T)


def _loss(p, loc, T, image, target, wt):
    r = _predict(p, loc, T, image) - target
    return float(np.sum(wt * (r.real ** 2 + r.imag ** 2)))


def _grad(p, loc, T, image, target, wt):
    """2 Re(M^H W r), M = degrid o IMAGE_TO_GRID, M^H = GRID_TO_IMAGE / n^2 o grid."""
    r = _predict(p, loc, T, image) - target
    G = O.grid_separable(p, loc, wt * r, None, T)
    l = O.pixel_l(p.N, p.fov)
    L, M = np.meshgrid(l, l)
    n2 = 1 - L * L - M * M
    return 2 * np.real(O.grid_to_image(p, G) / n2)


def test_oracle_chi2_gradient_matches_central_differences():
    p = O.Params(32, math.radians(4.0), 8, 4, 5, 300.0)
    rng = np.random.default_rng(17)
    n = 300
    u = rng.uniform(-12, 12, n) / p.fov
    v = rng.uniform(-12, 12, n) / p.fov
    w = rng.uniform(-300, 300, n)
    loc = O.locate(p, u, v, w)
    T = O.taps(p)
    image = rng.standard_normal((32, 32))
    target = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    wt = rng.uniform(0.5, 1.0, n)
    g = _grad(p, loc, T, image, target, wt)
    h = 1e-3
    for _ in range(12):
        b, a = rng.integers(0, 32, 2)
        e = np.zeros((32, 32))
        e[b, a] = h
        fd = (_loss(p, loc, T, image + e, target, wt) -
              _loss(p, loc, T, image - e, target, wt)) / (2 * h)
        assert abs(fd - g[b, a]) <= 1e-7 * (abs(g[b, a]) + np.max(np.abs(g)) * 1e-3)
