"""sepw_grid_noalloc: gridding for callers that cannot allocate device memory
(for example a real-time pipeline that reserves its memory at start-up and
must not block on cudaMalloc while it observes, or a plugin whose host
framework owns the memory pool).  Call after call it must give the grid of the
FP64 oracle within the FP32 tolerance, and the same grid as sepw_grid (tiled
FP32 form), even though every call reuses the same fixed scratch array.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import oracle as O
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
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_grid(wl):
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    return O.grid_separable(p, loc, wl.vis, wl.weight, O.taps(p)), int((~loc["keep"]).sum())


def _run(torch, S, wl, form=None):
    # the caller's form does not matter: noalloc always runs the tiled form
    prm = S.make_params(**wl.params(), form=S.FORM_TILED if form is None else form)
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TILED))
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
    return got.cpu().numpy(), ref.cpu().numpy(), int(nd.item()), int(nd_ref.item())


def test_noalloc_matches_oracle_and_grid_on_two_calls(env):
    torch, S = env
    # two different workloads back to back: the second call must not see any
    # state left in the shared scratch by the first; the second names a
    # tensor-core form (ignored) with a support the tensor cores do not take
    a = synth.random_case(31, 9000, 256, 16, 16, 33, edge_fraction=0.1)
    b = synth.random_case(32, 4000, 160, 20, 8, 9, edge_fraction=0.1)
    for wl, form in ((a, None), (b, S.FORM_TC_BF16)):
        got, ref, nd, nd_ref = _run(torch, S, wl, form)
        want, nd_want = _oracle_grid(wl)
        assert _rel(got, want) <= TOL_FP32
        assert _rel(got, ref) <= TOL_FP32
        assert nd == nd_ref == nd_want and nd > 0


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


def test_noalloc_rejects_taps_not_16_byte_aligned(env):
    # checked on the host before anything is enqueued: nothing is launched
    torch, S = env
    wl = synth.random_case(34, 64, 64, 8, 4, 3)
    prm = S.make_params(**wl.params(), form=S.FORM_TILED)
    ntaps = wl.n_wplanes * wl.oversample * wl.support
    buf = torch.zeros(ntaps + 1, dtype=torch.complex64, device="cuda")
    taps = buf[1:]  # 8 bytes past a 16-byte boundary
    assert taps.data_ptr() % 16 == 8
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    grid = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    rc = S.sepw_grid_noalloc(prm, taps, d["u"], d["v"], d["w"], d["vis"], d["weight"], grid)
    assert rc == S.EINVAL
    assert float(grid.abs().sum()) == 0.0
