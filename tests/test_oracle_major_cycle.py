"""Pins of the oracle's least-squares major cycles (conjugate gradients on
the normal equations of prediction, preconditioned by the grid correction):
the dot-product test of the prediction operator against its adjoint, and the
algebraic invariants every CG run has to show (non-increasing chi^2,
orthogonal residuals, directions conjugate under the normal operator, the
first step an exact line search).  The operators themselves are pinned by the
pipeline tests (prediction integral, adjointness of the gridder)."""
import math

import numpy as np

import oracle as O


def _case(seed=1, n=600):
    p = O.Params(16, math.radians(4.0), 8, 8, 5, 200.0)
    rng = np.random.default_rng(seed)
    u = rng.uniform(-6, 6, n) / p.fov
    v = rng.uniform(-6, 6, n) / p.fov
    w = rng.uniform(-200, 200, n)
    loc = O.locate(p, u, v, w)
    vis = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    wt = rng.uniform(0.5, 1, n)
    return p, loc, O.taps(p), vis, wt, rng


def test_prediction_adjoint_dot_product():
    p, loc, T, _, _, rng = _case()
    x = rng.standard_normal((p.N, p.N)) + 1j * rng.standard_normal((p.N, p.N))
    y = rng.standard_normal(len(loc["keep"])) + 1j * rng.standard_normal(len(loc["keep"]))
    lhs = np.vdot(y, O.predict_op(p, loc, T, x))
    rhs = np.vdot(O.predict_adjoint(p, loc, T, y), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_cg_invariants():
    p, loc, T, vis, wt, _ = _case(2)
    x, losses, rs, ds = O.cg_major_cycles(p, loc, T, vis, wt, 12)
    losses = np.asarray(losses)
    assert np.all(np.diff(losses) <= 1e-12 * losses[0])
    assert losses[-1] < 0.95 * losses[0]
    R = np.array([r.ravel() for r in rs])
    G = R @ R.T
    nrm = np.sqrt(np.diag(G))
    assert np.max(np.abs(G / np.outer(nrm, nrm) - np.eye(len(rs)))) < 1e-8

    # CG runs on y, x = Dg y, with Dg = n c1 c1 (the grid correction)
    l = O.pixel_l(p.N, p.fov)
    L, M = np.meshgrid(l, l)
    c1 = O.kb_taper(O.pixel_nu(p.N), p.S, p.kb_beta)
    Dg = np.sqrt(1 - L * L - M * M) * c1[None, :] * c1[:, None]

    def normal(y):
        return Dg * O.predict_adjoint(p, loc, T, wt * O.predict_op(p, loc, T, Dg * y)).real

    D = np.array([d.ravel() for d in ds[:6]])
    Q = np.array([normal(d).ravel() for d in ds[:6]])
    C = D @ Q.T
    dn = np.sqrt(np.abs(np.diag(C)))
    off = np.abs(C / np.outer(dn, dn) - np.eye(6))
    assert np.max(off) < 1e-8
    # the first step is the exact line search along the negative gradient in y
    r0 = rs[0]
    assert np.max(np.abs(r0 - Dg * O.predict_adjoint(p, loc, T, wt * vis).real)) < \
        1e-12 * np.max(np.abs(r0))
    a0 = float(np.sum(r0 * r0)) / float(np.sum(r0 * normal(r0)))
    x1, _, _, _ = O.cg_major_cycles(p, loc, T, vis, wt, 1)
    assert np.max(np.abs(x1 - Dg * a0 * r0)) < 1e-12 * np.max(np.abs(x1))
