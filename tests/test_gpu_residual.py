"""Stored correction F_w - F~_w (Sec. 7) through the C ABI against the FP64
oracle: the table (float64 to 1e-10, float32 to its rounding), the
correction pass and its adjoint, and the separable pass plus the full
correction against the oracle's exact 2-D W-projection gridder."""
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
    return torch, S


def rel_l2(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case():
    return synth.random_case(111, 6000, 96, 8, 8, 5, w_max=800.0, fov=math.radians(6.0),
                             edge_fraction=0.05)


@pytest.fixture(scope="module")
def oracle_tables():
    wl = _case()
    p = O.params_from(wl.params())
    return wl, p, O.exact_table(p), O.taps(p)


@pytest.mark.parametrize("Sr,OSr", [(8, 8), (6, 4), (2, 2)])
def test_correction_table(env, oracle_tables, Sr, OSr):
    torch, S = env
    wl, p, K, T = oracle_tables
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TILED))
    want = O.residual_table(p, Sr, OSr, K=K, T=T)
    got = S.sepw_make_residual_f64(ctx, Sr, OSr).cpu().numpy()
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(K))
    g32 = S.sepw_make_residual(ctx, Sr, OSr).cpu().numpy()
    assert np.max(np.abs(g32 - got)) <= 2 ** -23 * np.max(np.abs(got)) + 1e-30


@pytest.mark.parametrize("form", ["tiled", "tc_fp16x2", "tc_bf16x2"])
def test_separable_plus_correction_is_exact_w_projection(env, oracle_tables, form):
    torch, S = env
    wl, p, K, T = oracle_tables
    f = {"tiled": S.FORM_TILED, "tc_fp16x2": S.FORM_TC_FP16X2,
         "tc_bf16x2": S.FORM_TC_BF16X2}[form]
    ctx = S.sepw_create(S.make_params(**wl.params(), form=f))
    taps = S.sepw_make_taps(ctx)
    table = S.sepw_make_residual(ctx, p.S, p.OS)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    S.sepw_plan(ctx, d["u"], d["v"], d["w"])
    N = wl.grid_size
    grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S.sepw_grid_planned(ctx, taps, d["vis"], d["weight"], grid)
    S.sepw_grid_residual_planned(ctx, table, d["vis"], d["weight"], grid)
    loc = O.locate(p, wl.u, wl.v, wl.w)
    exact = O.grid_exact2d(p, loc, wl.vis, wl.weight, K)
    sep = O.grid_separable(p, loc, wl.vis, wl.weight, T)
    assert rel_l2(sep, exact) > 1e-5  # the correction matters at this bar
    assert rel_l2(grid.cpu().numpy(), exact) <= 1e-5
    # degridding: separable pass then the correction's adjoint
    rng = np.random.default_rng(5)
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    Xd = torch.from_numpy(X).cuda()
    out = torch.empty(wl.nvis, dtype=torch.complex64, device="cuda")
    S.sepw_degrid_planned(ctx, taps, Xd, d["weight"], out)
    S.sepw_degrid_residual_planned(ctx, table, Xd, d["weight"], out)
    R = O.residual_table(p, K=K, T=T)
    want = O.degrid_separable(p, loc, X, wl.weight, T)
    O.degrid_residual(p, loc, X, wl.weight, R, out=want)
    assert rel_l2(out.cpu().numpy(), want) <= 1e-5


def test_truncated_correction_pass(env, oracle_tables):
    torch, S = env
    wl, p, K, T = oracle_tables
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TILED))
    table = S.sepw_make_residual(ctx, 6, 4)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    S.sepw_plan(ctx, d["u"], d["v"], d["w"])
    N = wl.grid_size
    grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S.sepw_grid_residual_planned(ctx, table, d["vis"], d["weight"], grid)
    loc = O.locate(p, wl.u, wl.v, wl.w)
    want = O.grid_residual(p, loc, wl.vis, wl.weight, O.residual_table(p, 6, 4, K=K, T=T))
    assert rel_l2(grid.cpu().numpy(), want) <= 1e-5


def test_correction_rejects(env):
    torch, S = env
    wl = _case()
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_PLAIN))
    for Sr, OSr in ((3, 8), (10, 8), (8, 3)):
        with pytest.raises(S.SepwError) as e:
            S.sepw_make_residual(ctx, Sr, OSr)
        assert e.value.status == S.EINVAL
    table = S.sepw_make_residual(ctx, 8, 8)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis")}
    S.sepw_plan(ctx, d["u"], d["v"], d["w"])
    grid = torch.zeros((96, 96), dtype=torch.complex64, device="cuda")
    with pytest.raises(S.SepwError) as e:
        S.sepw_grid_residual_planned(ctx, table, d["vis"], None, grid)
    assert e.value.status == S.ENOTSUP
