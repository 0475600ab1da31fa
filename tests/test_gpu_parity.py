"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: bit-exact for cell, oversample and plane indices and the conjugation
and keep flags; float64 taps within 1e-12 of the oracle relative to the
largest tap; float32 taps within one float32 rounding of the oracle's values;
grids and predicted visibilities within relative L2 1e-5 for the FP32 forms
(the tolerance stated for the FP32 form).  Inputs are the seeded synthetic
workloads of ``synth``.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_07152_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def S_():
    import paper_1511_07152_gb300.sepw as S
    return S


def _ctx(S, wl, form, tile=0):
    prm = S.make_params(**wl.params(), tile=tile, form=form)
    return S.sepw_create(prm)


def _dev(torch, wl):
    d = dict(u=torch.from_numpy(wl.u).cuda(), v=torch.from_numpy(wl.v).cuda(),
             w=torch.from_numpy(wl.w).cuda(),
             vis=torch.from_numpy(wl.vis).cuda(),
             weight=torch.from_numpy(wl.weight).cuda())
    return d


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


CASES = {
    "small_disk": lambda: synth.small_disk(),
    "rand_S8": lambda: synth.random_case(1, 6000, 128, 8, 8, 9, edge_fraction=0.1),
    "rand_S12": lambda: synth.random_case(2, 6000, 160, 12, 16, 17, edge_fraction=0.1),
    "rand_S16": lambda: synth.random_case(3, 8000, 256, 16, 16, 33, edge_fraction=0.1),
    "rand_S16_P1": lambda: synth.random_case(4, 3000, 96, 16, 4, 1, edge_fraction=0.1),
    "rand_S2_OS1": lambda: synth.random_case(5, 3000, 64, 2, 1, 3, edge_fraction=0.1),
    # supports 4, 8, 12, 16 take the register-block kernels, the others the
    # column-per-lane kernels
    "rand_S4": lambda: synth.random_case(6, 3000, 64, 4, 8, 5, edge_fraction=0.1),
    "rand_S10": lambda: synth.random_case(7, 4000, 128, 10, 8, 9, edge_fraction=0.1),
    "rand_S20": lambda: synth.random_case(8, 4000, 192, 20, 8, 9, edge_fraction=0.1),
}


# --------------------------------------------------------------------------
# taps
# --------------------------------------------------------------------------


@pytest.mark.parametrize("name", ["small_disk", "rand_S12", "rand_S16_P1", "rand_S2_OS1"])
def test_taps_f64_and_f32(torch_cuda, S_, name):
    torch = torch_cuda
    wl = CASES[name]()
    ctx = _ctx(S_, wl, S_.FORM_TILED)
    want = O.taps(O.params_from(wl.params()))
    got64 = S_.sepw_make_taps_f64(ctx).cpu().numpy()
    assert np.max(np.abs(got64 - want)) <= 1e-12 * np.max(np.abs(want))
    got32 = S_.sepw_make_taps(ctx).cpu().numpy()
    w32 = want.astype(np.complex64)
    # one float32 rounding of float64 values that agree to 1e-12
    ulp = np.spacing(np.maximum(np.abs(w32.real), np.abs(w32.imag)).astype(np.float32))
    slack = ulp + 2e-12 * np.max(np.abs(want))
    assert np.all(np.abs(got32.real.astype(np.float64) - w32.real) <= slack)
    assert np.all(np.abs(got32.imag.astype(np.float64) - w32.imag) <= slack)
    torch.cuda.synchronize()


def test_taps_meerkat_scale(torch_cuda, S_):
    """Full-size table of the 32M-visibility workload (P=128, OS=16, S=16,
    N=4096), float64 parity."""
    p = dict(grid_size=4096, fov=math.radians(1.0), support=16, oversample=16,
             n_wplanes=128, w_max=31000.0, gamma=5 / 24, kb_beta=2.34 * 16)
    ctx = S_.sepw_create(S_.make_params(**p))
    want = O.taps(O.Params(**p))
    got = S_.sepw_make_taps_f64(ctx).cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


# --------------------------------------------------------------------------
# locate
# --------------------------------------------------------------------------


@pytest.mark.parametrize("name", list(CASES))
def test_locate_bit_exact(torch_cuda, S_, name):
    torch = torch_cuda
    wl = CASES[name]()
    u, v, w = wl.u.copy(), wl.v.copy(), wl.w.copy()
    # non-finite coordinates and w exactly on a plane boundary
    u[:3] = [np.nan, np.inf, -np.inf]
    w[3:6] = [np.nan, -0.0, wl.w_max]
    v[6] = np.nan
    ctx = _ctx(S_, wl, S_.FORM_TILED)
    out = S_.sepw_locate(ctx, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(),
                         torch.from_numpy(w).cuda())
    want = O.locate(O.params_from(wl.params()), u, v, w)
    for k in ("cu", "cv", "ou", "ov", "plane"):
        assert np.array_equal(out[k].cpu().numpy(), want[k]), k
    assert np.array_equal(out["conj"].cpu().numpy().astype(bool), want["conj"])
    assert np.array_equal(out["keep"].cpu().numpy().astype(bool), want["keep"])
    assert 0 < want["keep"].sum() < len(u) or name == "small_disk"


@pytest.mark.parametrize("N,OS", [(4096, 16), (256, 8), (1000, 4), (96, 16)])
def test_locate_rounding_boundaries(torch_cuda, S_, N, OS):
    """Coordinates whose scaled position y OS + 1/2 (y = u fov) lies within a
    few ulps of an integer, both sides, or whose sum y + N/2 rounds at its
    last bit, over the whole grid and beyond its edges: every result, whether
    the locate takes its integer path or falls back to FP64 arithmetic,
    equals the oracle's bit for bit."""
    torch = torch_cuda
    rng = np.random.default_rng(17)
    fov = math.radians(1.0)
    H = N // 2
    ys = []
    for k in rng.integers(-H * OS - 4 * OS, H * OS + 4 * OS, 3000):
        y = (float(k) - 0.5) / OS
        up = dn = y
        ys.append(y)
        for _ in range(4):
            up = float(np.nextafter(up, np.inf))
            dn = float(np.nextafter(dn, -np.inf))
            ys += [up, dn]
    for k in rng.integers(1, 1 << 40, 3000):
        ys.append(float(k) * 2.0 ** (int(rng.integers(-20, 12)) - 40) - H)
    ys += list(rng.uniform(-H - 8, H + 8, 20000))
    ys += [0.0, -0.0, 5e-324, -5e-324, float(H), -float(H), 0.5 / OS, -0.5 / OS]
    y = np.array(ys)
    n = len(y)
    u = y / fov
    v = rng.permutation(y) / fov
    w = rng.uniform(-300.0, 300.0, n)
    p = dict(grid_size=N, fov=fov, support=8, oversample=OS, n_wplanes=9, w_max=300.0)
    ctx = S_.sepw_create(S_.make_params(**p, form=S_.FORM_TILED))
    out = S_.sepw_locate(ctx, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(),
                         torch.from_numpy(w).cuda())
    want = O.locate(O.Params(**p), u, v, w)
    for k in ("cu", "cv", "ou", "ov", "plane"):
        assert np.array_equal(out[k].cpu().numpy(), want[k]), k
    assert np.array_equal(out["keep"].cpu().numpy().astype(bool), want["keep"])
    assert 0 < want["keep"].sum() < n


def test_locate_meerkat_full_bit_exact(torch_cuda, S_):
    """All 32,256,000 visibilities of the full-size workload."""
    torch = torch_cuda
    wl = synth.meerkat_like()
    ctx = _ctx(S_, wl, S_.FORM_TILED)
    out = S_.sepw_locate(ctx, torch.from_numpy(wl.u).cuda(), torch.from_numpy(wl.v).cuda(),
                         torch.from_numpy(wl.w).cuda())
    want = O.locate(O.params_from(wl.params()), wl.u, wl.v, wl.w)
    for k in ("cu", "cv", "ou", "ov", "plane"):
        assert np.array_equal(out[k].cpu().numpy(), want[k]), k
    assert np.array_equal(out["conj"].cpu().numpy().astype(bool), want["conj"])
    assert np.array_equal(out["keep"].cpu().numpy().astype(bool), want["keep"])


# --------------------------------------------------------------------------
# gridding / degridding against the FP64 oracle
# --------------------------------------------------------------------------


def _oracle_grid(wl):
    p = O.params_from(wl.params())
    T = O.taps(p)
    loc = O.locate(p, wl.u, wl.v, wl.w)
    return O.grid_separable(p, loc, wl.vis, wl.weight, T), loc, T, p


FORMS = ["plain", "tiled"]


def _form(S, name):
    return S.FORM_PLAIN if name == "plain" else S.FORM_TILED


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", list(CASES))
def test_grid_parity(torch_cuda, S_, form, name):
    torch = torch_cuda
    wl = CASES[name]()
    want, loc, _, _ = _oracle_grid(wl)
    ctx = _ctx(S_, wl, _form(S_, form))
    taps = S_.sepw_make_taps(ctx)
    d = _dev(torch, wl)
    N = wl.grid_size
    grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    nd = torch.zeros(1, dtype=torch.int64, device="cuda")
    S_.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], grid, nd)
    got = grid.cpu().numpy()
    assert rel_l2(got, want) <= TOL_FP32
    assert int(nd.item()) == int((~loc["keep"]).sum())


@pytest.mark.parametrize("tile", [8, 16, 32, 48])
def test_grid_tiled_tile_sizes(torch_cuda, S_, tile):
    torch = torch_cuda
    wl = CASES["rand_S16"]()
    if tile + wl.support - 1 > 64:
        pytest.skip("window too large")
    want, _, _, _ = _oracle_grid(wl)
    ctx = _ctx(S_, wl, S_.FORM_TILED, tile=tile)
    taps = S_.sepw_make_taps(ctx)
    d = _dev(torch, wl)
    N = wl.grid_size
    grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S_.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], grid)
    assert rel_l2(grid.cpu().numpy(), want) <= TOL_FP32


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name", list(CASES))
def test_degrid_parity(torch_cuda, S_, form, name):
    torch = torch_cuda
    wl = CASES[name]()
    p = O.params_from(wl.params())
    T = O.taps(p)
    loc = O.locate(p, wl.u, wl.v, wl.w)
    rng = np.random.default_rng(99)
    N = wl.grid_size
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    want = O.degrid_separable(p, loc, X, wl.weight, T)
    ctx = _ctx(S_, wl, _form(S_, form))
    taps = S_.sepw_make_taps(ctx)
    d = _dev(torch, wl)
    out = torch.full((wl.nvis,), complex(7, 7), dtype=torch.complex64, device="cuda")
    S_.sepw_degrid(ctx, taps, d["u"], d["v"], d["w"], torch.from_numpy(X).cuda(),
                   d["weight"], out)
    got = out.cpu().numpy()
    assert rel_l2(got, want) <= TOL_FP32
    assert np.all(got[~loc["keep"]] == 0)


def test_heavy_tile_and_duplicates(torch_cuda, S_):
    """Many visibilities at one position (one tile holds several work items
    and one origin spans several warps), plus exact duplicates."""
    torch = torch_cuda
    n = 20000
    rng = np.random.default_rng(3)
    fov = math.radians(2.0)
    u = np.concatenate([np.full(n // 2, 3.3 / fov), rng.uniform(-5, 5, n // 2) / fov])
    v = np.concatenate([np.full(n // 2, -1.7 / fov), rng.uniform(-5, 5, n // 2) / fov])
    w = rng.uniform(-300, 300, n)
    vis = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    wt = rng.uniform(0.5, 1, n).astype(np.float32)
    wl = synth.Workload("heavy", 64, fov, 16, 16, 9, 300.0, u, v, w, vis, wt)
    want, _, _, _ = _oracle_grid(wl)
    for form in (S_.FORM_PLAIN, S_.FORM_TILED):
        ctx = _ctx(S_, wl, form)
        taps = S_.sepw_make_taps(ctx)
        d = _dev(torch, wl)
        grid = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
        S_.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], grid)
        assert rel_l2(grid.cpu().numpy(), want) <= TOL_FP32


def test_empty_single_and_all_dropped(torch_cuda, S_):
    torch = torch_cuda
    wl = CASES["rand_S8"]()
    for form in (S_.FORM_PLAIN, S_.FORM_TILED):
        ctx = _ctx(S_, wl, form)
        taps = S_.sepw_make_taps(ctx)
        N = wl.grid_size
        grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
        e = torch.empty(0, dtype=torch.float64, device="cuda")
        ev = torch.empty(0, dtype=torch.complex64, device="cuda")
        S_.sepw_grid(ctx, taps, e, e, e, ev, None, grid)
        assert float(grid.abs().sum()) == 0.0
        # one visibility
        one = lambda a: torch.from_numpy(np.ascontiguousarray(a[:1])).cuda()  # noqa: E731
        want, _, _, _ = _oracle_grid(synth.Workload("one", N, wl.fov, wl.support,
                                                    wl.oversample, wl.n_wplanes, wl.w_max,
                                                    wl.u[:1], wl.v[:1], wl.w[:1],
                                                    wl.vis[:1], wl.weight[:1]))
        S_.sepw_grid(ctx, taps, one(wl.u), one(wl.v), one(wl.w), one(wl.vis),
                     one(wl.weight), grid)
        assert rel_l2(grid.cpu().numpy(), want) <= TOL_FP32
        # everything dropped
        far = torch.full((100,), 1e12, dtype=torch.float64, device="cuda")
        nd = torch.zeros(1, dtype=torch.int64, device="cuda")
        g2 = torch.zeros_like(grid)
        S_.sepw_grid(ctx, taps, far, far, far, torch.ones(100, dtype=torch.complex64,
                                                             device="cuda"), None, g2, nd)
        assert int(nd.item()) == 100 and float(g2.abs().sum()) == 0.0
        out = torch.ones(100, dtype=torch.complex64, device="cuda")
        S_.sepw_degrid(ctx, taps, far, far, far, grid, None, out)
        assert float(out.abs().sum()) == 0.0


def test_plan_reuse_and_accumulate(torch_cuda, S_):
    """One plan serves several calls; sepw_grid accumulates into the grid."""
    torch = torch_cuda
    wl = CASES["rand_S16"]()
    want, loc, _, _ = _oracle_grid(wl)
    ctx = _ctx(S_, wl, S_.FORM_TILED)
    taps = S_.sepw_make_taps(ctx)
    d = _dev(torch, wl)
    S_.sepw_plan(ctx, d["u"], d["v"], d["w"])
    assert S_.sepw_plan_dropped(ctx) == int((~loc["keep"]).sum())
    N = wl.grid_size
    grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S_.sepw_grid_planned(ctx, taps, d["vis"], d["weight"], grid)
    S_.sepw_grid_planned(ctx, taps, d["vis"], d["weight"], grid)
    assert rel_l2(grid.cpu().numpy(), 2 * want) <= TOL_FP32
    o1 = torch.empty(wl.nvis, dtype=torch.complex64, device="cuda")
    o2 = torch.empty_like(o1)
    S_.sepw_degrid_planned(ctx, taps, grid, d["weight"], o1)
    S_.sepw_degrid_planned(ctx, taps, grid, d["weight"], o2)
    assert torch.equal(o1, o2)


def test_adjoint_identity_gpu(torch_cuda, S_):
    """<grid(V), X> = <V, degrid(X)> through the CUDA path (FP32)."""
    torch = torch_cuda
    wl = CASES["rand_S12"]()
    ctx = _ctx(S_, wl, S_.FORM_TILED)
    taps = S_.sepw_make_taps(ctx)
    d = _dev(torch, wl)
    N = wl.grid_size
    rng = np.random.default_rng(5)
    X = torch.from_numpy((rng.standard_normal((N, N)) +
                          1j * rng.standard_normal((N, N))).astype(np.complex64)).cuda()
    G = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S_.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], G)
    D = torch.empty(wl.nvis, dtype=torch.complex64, device="cuda")
    S_.sepw_degrid(ctx, taps, d["u"], d["v"], d["w"], X, d["weight"], D)
    lhs = np.vdot(G.cpu().numpy().astype(np.complex128), X.cpu().numpy())
    rhs = np.vdot(wl.vis.astype(np.complex128), D.cpu().numpy())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


# --------------------------------------------------------------------------
# image step
# --------------------------------------------------------------------------


@pytest.mark.parametrize("direction", [0, 1])
def test_image_step(torch_cuda, S_, direction):
    torch = torch_cuda
    wl = CASES["rand_S8"]()
    p = O.params_from(wl.params())
    N = wl.grid_size
    rng = np.random.default_rng(11)
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    if direction == 0:
        want = O.grid_to_image(p, X)
    else:
        want = O.image_to_grid(p, X)
    ctx = _ctx(S_, wl, S_.FORM_TILED)
    buf = torch.from_numpy(X.copy()).cuda()
    S_.sepw_image(ctx, direction, buf)
    got = buf.cpu().numpy()
    # compare where the correction 1/c1 does not amplify FFT rounding by more
    # than 1e3: |nu| < 0.35 on both axes for this taper
    nu = O.pixel_nu(N)
    inner = np.abs(nu) < 0.35
    if direction == 0:
        m = np.ix_(inner, inner)
        assert rel_l2(got[m], want[m]) <= 1e-5
    else:
        assert rel_l2(got, want) <= 1e-5


# --------------------------------------------------------------------------
# full-size workload (32,256,000 visibilities, 4096^2 grid)
# --------------------------------------------------------------------------


@pytest.fixture(scope="module")
def meerkat():
    return synth.meerkat_like()


def test_meerkat_grid_subsample_vs_oracle(torch_cuda, S_, meerkat):
    """1% seeded subsample of the full workload on the full 4096^2 grid, both
    forms, against the FP64 oracle."""
    torch = torch_cuda
    wl = meerkat.subsample(meerkat.nvis // 100)
    want, _, _, _ = _oracle_grid(wl)
    for form in (S_.FORM_PLAIN, S_.FORM_TILED):
        ctx = _ctx(S_, wl, form)
        taps = S_.sepw_make_taps(ctx)
        d = _dev(torch, wl)
        grid = torch.zeros((4096, 4096), dtype=torch.complex64, device="cuda")
        S_.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], grid)
        assert rel_l2(grid.cpu().numpy(), want) <= TOL_FP32


def _oracle_threads(p, wl, T, model=None):
    """The oracle on all visibilities of wl over the host's cores: contiguous
    shards per thread (its C loops release the interpreter lock), the shards'
    grids summed; with a model grid, each shard's predictions instead."""
    import concurrent.futures as cf
    import os
    nt = os.cpu_count() or 1
    q, r = divmod(wl.nvis, nt)
    bounds = [(k * q + min(k, r), (k + 1) * q + min(k + 1, r)) for k in range(nt)]

    def run(k):
        lo, hi = bounds[k]
        loc = O.locate(p, wl.u[lo:hi], wl.v[lo:hi], wl.w[lo:hi])
        if model is None:
            return O.grid_separable(p, loc, wl.vis[lo:hi], wl.weight[lo:hi], T)
        return O.degrid_separable(p, loc, model, wl.weight[lo:hi], T)

    with cf.ThreadPoolExecutor(nt) as ex:
        parts = list(ex.map(run, range(nt)))
    if model is None:
        total = parts[0]
        for g in parts[1:]:
            total += g
        return total
    return np.concatenate(parts)


def test_meerkat_full_size(torch_cuda, S_, meerkat):
    """All 32,256,000 visibilities in the benchmark's launch configuration
    (tiled form, plan + grid + degrid) against the FP64 oracle on all of them
    (run over the host's cores): the grid and every prediction within the
    FP32 bar; the BF16 hi + lo tensor-core form's grid and predictions at the
    same bar, the BF16 form's at 1e-2.  Also: the plain form's grid agrees,
    and gridding is linear (the sum of the grids of the two halves)."""
    torch = torch_cuda
    wl = meerkat
    N = 4096
    d = _dev(torch, wl)
    ctx_t = _ctx(S_, wl, S_.FORM_TILED)
    ctx_p = _ctx(S_, wl, S_.FORM_PLAIN)
    taps = S_.sepw_make_taps(ctx_t)
    gt = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S_.sepw_plan(ctx_t, d["u"], d["v"], d["w"])
    S_.sepw_grid_planned(ctx_t, taps, d["vis"], d["weight"], gt)
    # degrid the gridded image (a realistic model grid)
    out = torch.empty(wl.nvis, dtype=torch.complex64, device="cuda")
    S_.sepw_degrid_planned(ctx_t, taps, gt, d["weight"], out)
    a = gt.cpu().numpy()
    p = O.params_from(wl.params())
    T = O.taps(p)
    want = _oracle_threads(p, wl, T)
    assert rel_l2(a, want) <= TOL_FP32
    pred = _oracle_threads(p, wl, T, model=a.astype(np.complex128))
    assert rel_l2(out.cpu().numpy(), pred) <= TOL_FP32
    # the tensor-core forms on the same full workload and model grid: BF16
    # hi + lo at the FP32 bar, BF16 at its own (operand rounding 2^-8)
    for form, tol in ((S_.FORM_TC_BF16X2, TOL_FP32), (S_.FORM_TC_BF16, 1e-2)):
        ctx_c = _ctx(S_, wl, form)
        gc = torch.zeros_like(gt)
        S_.sepw_plan(ctx_c, d["u"], d["v"], d["w"])
        S_.sepw_grid_planned(ctx_c, taps, d["vis"], d["weight"], gc)
        assert rel_l2(gc.cpu().numpy(), want) <= tol, form
        S_.sepw_degrid_planned(ctx_c, taps, gt, d["weight"], out)
        assert S_.sepw_device_status(ctx_c) == S_.OK
        assert rel_l2(out.cpu().numpy(), pred) <= tol, form
        ctx_c.close()
        del gc
    del want, pred
    gp = torch.zeros_like(gt)
    S_.sepw_grid(ctx_p, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], gp)
    assert rel_l2(a, gp.cpu().numpy()) <= TOL_FP32
    h = wl.nvis // 2
    g2 = torch.zeros_like(gt)
    for sl in (slice(0, h), slice(h, None)):
        S_.sepw_grid(ctx_t, taps, d["u"][sl].contiguous(), d["v"][sl].contiguous(),
                     d["w"][sl].contiguous(), d["vis"][sl].contiguous(),
                     d["weight"][sl].contiguous(), g2)
    assert rel_l2(g2.cpu().numpy(), a) <= TOL_FP32


def test_full_step_graph_replay_matches_eager(torch_cuda, S_):
    """The whole planned step (zero, plan, grid, degrid) captured in one CUDA
    graph: two replays give the eager step's grid and predictions (to FP32
    rounding: the atomics' order may differ) and the oracle's within the FP32
    bar."""
    torch, S = torch_cuda, S_
    wl = synth.small_disk()
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TILED))
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    N = wl.grid_size
    grid = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    out = torch.empty(wl.nvis, dtype=torch.complex64, device="cuda")

    def step():
        grid.zero_()
        S.sepw_plan(ctx, d["u"], d["v"], d["w"])
        S.sepw_grid_planned(ctx, taps, d["vis"], d["weight"], grid)
        S.sepw_degrid_planned(ctx, taps, grid, d["weight"], out)

    step()
    torch.cuda.synchronize()
    g_eager, o_eager = grid.clone(), out.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        step()
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    want = O.grid_separable(p, loc, wl.vis, wl.weight, O.taps(p))
    for _ in range(2):
        grid.fill_(7.0)
        graph.replay()
        torch.cuda.synchronize()
        assert rel_l2(grid.cpu().numpy(), g_eager.cpu().numpy()) <= 1e-6
        assert rel_l2(out.cpu().numpy(), o_eager.cpu().numpy()) <= 1e-6
        assert rel_l2(grid.cpu().numpy(), want) <= TOL_FP32
    assert S.sepw_device_status(ctx) == S.OK


@pytest.mark.parametrize("chunk,parts", [(64, 1), (256, 3), (1024, 16), (2048, 0)])
def test_schedule_does_not_change_the_grid(torch_cuda, S_, chunk, parts):
    """Work items of any size and any split of them among the gridder's warps
    give the oracle's grid and predictions (FP32 rounding order aside)."""
    torch = torch_cuda
    wl = synth.random_case(81, 30000, 256, 16, 16, 33, edge_fraction=0.1,
                           radius_cells=40.0)  # dense tiles: many items per tile
    ctx = _ctx(S_, wl, S_.FORM_TILED)
    S_.sepw_set_schedule(ctx, chunk, parts)
    taps = S_.sepw_make_taps(ctx)
    d = _dev(torch, wl)
    N = wl.grid_size
    g = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    S_.sepw_plan(ctx, d["u"], d["v"], d["w"])
    S_.sepw_grid_planned(ctx, taps, d["vis"], d["weight"], g)
    out = torch.empty(wl.nvis, dtype=torch.complex64, device="cuda")
    S_.sepw_degrid_planned(ctx, taps, g, d["weight"], out)
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    T = O.taps(p)
    a = g.cpu().numpy()
    assert rel_l2(a, O.grid_separable(p, loc, wl.vis, wl.weight, T)) <= TOL_FP32
    assert rel_l2(out.cpu().numpy(),
                  O.degrid_separable(p, loc, a.astype(np.complex128), wl.weight, T)) <= TOL_FP32


def test_schedule_rejects_bad_sizes(torch_cuda, S_):
    wl = synth.random_case(82, 100, 64, 8, 4, 3)
    ctx = _ctx(S_, wl, S_.FORM_TILED)
    for chunk, parts in ((32, 0), (4096, 0), (100, 0), (2048, 17), (2048, -1)):
        with pytest.raises(S_.SepwError):
            S_.sepw_set_schedule(ctx, chunk, parts)
