"""sepw_grid_noalloc: gridding for callers that cannot allocate device memory
(for example a real-time pipeline that reserves its memory at start-up, or a
plugin whose host framework owns the memory pool).  It must give the same grid
as sepw_grid (tiled FP32 form) within the FP32 tolerance, call after call,
even though every call reuses the same fixed scratch array.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_07152_gb300 import build
    build.build()
    import paper_1511_07152_gb300.sepw as S
    return torch, S


def _rel(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(torch, S, wl, tile=0):
    prm = S.make_params(**wl.params(), tile=tile, form=S.FORM_TILED)
    ctx = S.sepw_create(prm)
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    N = wl.grid_size
    ref = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
    nd_ref = torch.zeros(1, dtype=torch.int64, device="cuda")
    S.sepw_grid(ctx, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], ref, nd_ref)
    got = torch.zeros_like(ref)
    nd = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    rc = S.sepw_grid_noalloc(prm, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"],
                             got, nd)
    torch.cuda.synchronize()
    assert rc == S.OK
    return got, ref, int(nd.item()), int(nd_ref.item())


def test_noalloc_matches_grid_on_two_calls(env):
    torch, S = env
    # two different workloads back to back: the second call must not see any
    # state left in the shared scratch by the first
    a = synth.random_case(31, 9000, 256, 16, 16, 33, edge_fraction=0.1)
    b = synth.random_case(32, 4000, 160, 12, 8, 9, edge_fraction=0.1)
    for wl in (a, b):
        got, ref, nd, nd_ref = _run(torch, S, wl)
        assert _rel(got, ref) <= TOL_FP32
        assert nd == nd_ref and nd > 0


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, S = env
    wl = synth.random_case(33, 16, 64, 8, 4, 3)
    prm = S.make_params(**wl.params(), form=S.FORM_TILED)
    ctx = S.sepw_create(prm)
    taps = S.sepw_make_taps(ctx)
    n = S.NOALLOC_MAX_VIS + 1
    big = torch.zeros(n, dtype=torch.float64, device="cuda")
    vis = torch.zeros(n, dtype=torch.complex64, device="cuda")
    grid = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    assert S.sepw_grid_noalloc(prm, taps, big, big, big, vis, None, grid) == S.ETOOLARGE
    # a grid whose tile count exceeds the scratch is refused too
    prm2 = S.make_params(grid_size=8192, fov=0.02, support=8, oversample=4, n_wplanes=3,
                         w_max=100.0, tile=8, form=S.FORM_TILED)
    g2 = torch.zeros((8192, 8192), dtype=torch.complex64, device="cuda")
    t2 = torch.zeros((3, 4, 8), dtype=torch.complex64, device="cuda")
    small = torch.zeros(4, dtype=torch.float64, device="cuda")
    sv = torch.zeros(4, dtype=torch.complex64, device="cuda")
    assert S.sepw_grid_noalloc(prm2, t2, small, small, small, sv, None, g2) == S.ETOOLARGE
    assert float(g2.abs().sum()) == 0.0
