"""Batched gridding (many W-stacking layers / channels, Sec. 4.3) in one
persistent launch, against per-grid gridding and the FP64 oracle; CUDA-graph
capture and replay of the planned launch; the autotuner on the GPU."""
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


def _batch(seed=0, ngrids=7, N=128, S_=12):
    """Uneven counts (one grid empty), residual w per layer, seeded."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(200, 4000, ngrids)
    counts[2] = 0
    fov = math.radians(2.0)
    parts = []
    for g, n in enumerate(counts):
        parts.append(synth.random_case(200 + g, int(n), N, S_, 8, 9, w_max=400.0, fov=fov))
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    cat = lambda k: np.concatenate([getattr(p, k) for p in parts])  # noqa: E731
    wl = synth.Workload("batch", N, fov, S_, 8, 9, 400.0, cat("u"), cat("v"), cat("w"),
                        cat("vis"), cat("weight"))
    return wl, offs, parts


def rel_l2(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("form,tol", [(1, 1e-5), (3, 1.5e-3), (0, 1e-5), (2, 1e-2), (5, 1e-5),
                                      (6, 1.5e-3)])
def test_batched_matches_oracle_per_grid(env, form, tol):
    torch, S = env
    wl, offs, parts = _batch()
    ctx = S.sepw_create(S.make_params(**wl.params(), form=form))
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    ng = len(offs) - 1
    N = wl.grid_size
    grids = torch.zeros((ng, N, N), dtype=torch.complex64, device="cuda")
    nd = torch.zeros(1, dtype=torch.int64, device="cuda")
    S.sepw_grid_batched(ctx, taps, offs, d["u"], d["v"], d["w"], d["vis"], d["weight"],
                        grids, nd)
    got = grids.cpu().numpy()
    p = O.params_from(wl.params())
    T = O.taps(p)
    ndrop = 0
    for g, part in enumerate(parts):
        loc = O.locate(p, part.u, part.v, part.w)
        ndrop += int((~loc["keep"]).sum())
        want = O.grid_separable(p, loc, part.vis, part.weight, T)
        if part.nvis == 0:
            assert float(np.abs(got[g]).sum()) == 0.0
        else:
            assert rel_l2(got[g], want) <= tol, g
    if form != 0:
        assert int(nd.item()) == ndrop


def test_batched_degrid_and_graph_replay(env):
    """The planned batched launch captured in a CUDA graph and replayed
    twice gives twice the grid; batched degridding matches the oracle."""
    torch, S = env
    wl, offs, parts = _batch(seed=1)
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TILED))
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    ng = len(offs) - 1
    N = wl.grid_size
    S.sepw_plan_batched(ctx, offs, d["u"], d["v"], d["w"])
    ref = torch.zeros((ng, N, N), dtype=torch.complex64, device="cuda")
    S.sepw_grid_planned(ctx, taps, d["vis"], d["weight"], ref)
    grids = torch.zeros_like(ref)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        S.sepw_grid_planned(ctx, taps, d["vis"], d["weight"], grids, stream=s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert rel_l2(grids.cpu().numpy(), 2 * ref.cpu().numpy()) <= 1e-5
    # degridding of the batch from random model grids
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((ng, N, N)) + 1j * rng.standard_normal((ng, N, N))
         ).astype(np.complex64)
    out = torch.empty(wl.nvis, dtype=torch.complex64, device="cuda")
    S.sepw_degrid_planned(ctx, taps, torch.from_numpy(X).cuda(), d["weight"], out)
    got = out.cpu().numpy()
    p = O.params_from(wl.params())
    T = O.taps(p)
    for gi, part in enumerate(parts):
        if part.nvis == 0:
            continue
        loc = O.locate(p, part.u, part.v, part.w)
        want = O.degrid_separable(p, loc, X[gi], part.weight, T)
        assert rel_l2(got[offs[gi]:offs[gi + 1]], want) <= 1e-5


@pytest.mark.parametrize("form,tol", [(2, 1e-2), (3, 1.5e-3), (4, 1e-5), (5, 1e-5), (6, 1.5e-3)])
def test_batched_tc_degrid_matches_oracle_per_grid(env, form, tol):
    """Degridding a batched plan in the tensor-core forms (BF16, FP16 and
    their hi + lo splits on the contraction degridder, whose windows carry
    each grid's base offset; TF32 on the tiled FP32 degridder): per-grid
    predictions against the oracle at the form's bar, the empty grid
    included."""
    torch, S = env
    wl, offs, parts = _batch(seed=4)
    ctx = S.sepw_create(S.make_params(**wl.params(), form=form))
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    ng = len(offs) - 1
    N = wl.grid_size
    S.sepw_plan_batched(ctx, offs, d["u"], d["v"], d["w"])
    rng = np.random.default_rng(5)
    X = (rng.standard_normal((ng, N, N)) + 1j * rng.standard_normal((ng, N, N))
         ).astype(np.complex64)
    out = torch.full((wl.nvis,), complex(7, 7), dtype=torch.complex64, device="cuda")
    S.sepw_degrid_planned(ctx, taps, torch.from_numpy(X).cuda(), d["weight"], out)
    assert S.sepw_device_status(ctx) == S.OK
    got = out.cpu().numpy()
    p = O.params_from(wl.params())
    T = O.taps(p)
    for gi, part in enumerate(parts):
        if part.nvis == 0:
            continue
        loc = O.locate(p, part.u, part.v, part.w)
        want = O.degrid_separable(p, loc, X[gi], part.weight, T)
        assert rel_l2(got[offs[gi]:offs[gi + 1]], want) <= tol, (form, gi)


def test_batched_rejects_bad_offsets(env):
    torch, S = env
    wl, offs, _ = _batch(seed=2, ngrids=3)
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TILED))
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w")}
    bad = offs.copy()
    bad[1], bad[2] = bad[2], bad[1]
    if bad[1] != bad[2]:
        with pytest.raises(S.SepwError):
            S.sepw_plan_batched(ctx, bad, d["u"], d["v"], d["w"])


def test_autotune_on_gpu(env, tmp_path):
    torch, S = env
    from paper_1511_07152_gb300 import autotune as A
    wl = synth.random_case(9, 20000, 256, 16, 16, 17)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    res = A.tune(wl.params(), d["u"], d["v"], d["w"], d["vis"], d["weight"], max_error=1e-5,
                 reps=2, cache_path=str(tmp_path / "t.json"))
    assert A.FORM_ERROR[res["form"]] <= 1e-5
    assert res["tile"] in A.candidate_tiles(16, res["form"])
    assert (res["chunk"], res["grid_parts"]) in A.candidate_schedules(res["form"])
    assert len(res["schedule_timings"]) == len(A.candidate_schedules(res["form"]))
    res2 = A.tune(wl.params(), d["u"], d["v"], d["w"], d["vis"], d["weight"],
                  max_error=1e-5, cache_path=str(tmp_path / "t.json"))
    assert res2 == res
