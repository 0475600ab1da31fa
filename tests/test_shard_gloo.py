"""Visibility-sharded gridding, degridding and W-stacking imaging over two
gloo ranks on the CPU (one process per rank, rendezvous on 127.0.0.1), with
the FP64 oracle as the per-shard function.  The all-reduced grid and image
must equal the oracle's single-process results on all visibilities (the
sums differ only in rounding order), and the gathered predictions must equal
the oracle's predictions of all visibilities exactly (the same arithmetic per
visibility, from the model grid that rank 0 broadcasts)."""
import math
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1511_07152_gb300 import shard as SH  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import synth
    return synth.random_case(61, 3001, 64, 8, 4, 5, w_max=300.0, fov=math.radians(4.0),
                             edge_fraction=0.1)


def _model(N):
    rng = np.random.default_rng(5)
    return rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))


CENTRES = [-200.0, 0.0, 200.0]


def _rank_main(rank, ws, port, result_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        wl = _case()
        p = O.params_from(wl.params())
        T = O.taps(p)
        lo, hi = SH.shard_bounds(wl.nvis, rank, ws)
        t = {k: torch.from_numpy(np.ascontiguousarray(getattr(wl, k)[lo:hi]))
             for k in ("u", "v", "w", "vis", "weight")}

        def grid_fn(u, v, w, vis, weight, grid):
            loc = O.locate(p, u.numpy(), v.numpy(), w.numpy())
            grid += torch.from_numpy(O.grid_separable(p, loc, vis.numpy(), weight.numpy(), T))

        def degrid_fn(u, v, w, grid, weight):
            loc = O.locate(p, u.numpy(), v.numpy(), w.numpy())
            return torch.from_numpy(O.degrid_separable(p, loc, grid.numpy(), weight.numpy(), T))

        def image_fn(u, v, w, vis, weight, image):
            image.copy_(torch.from_numpy(O.wstack_image(
                p, u.numpy(), v.numpy(), w.numpy(), vis.numpy(), weight.numpy(), CENTRES)))

        N = wl.grid_size
        grid = torch.zeros((N, N), dtype=torch.complex128)
        SH.grid_sharded(grid_fn, t["u"], t["v"], t["w"], t["vis"], t["weight"], grid)
        # only rank 0 holds the model; the others start from zeros
        model = torch.from_numpy(_model(N)) if rank == 0 else torch.zeros((N, N),
                                                                          dtype=torch.complex128)
        pred = SH.degrid_sharded(degrid_fn, t["u"], t["v"], t["w"], model, t["weight"],
                                 src=0, gather=True, n_total=wl.nvis)
        own = SH.degrid_sharded(degrid_fn, t["u"], t["v"], t["w"], model, t["weight"])
        image = torch.zeros((N, N), dtype=torch.complex128)
        SH.wstack_image_sharded(image_fn, t["u"], t["v"], t["w"], t["vis"], t["weight"], image)
        result_q.put((rank, grid.numpy(), pred.numpy(), own.numpy(), (lo, hi), image.numpy()))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_shard_bounds_partition():
    for n in (0, 1, 7, 3001, 32256000):
        for world in (1, 2, 3, 8):
            b = [SH.shard_bounds(n, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        SH.shard_bounds(5, 2, 2)


def test_two_gloo_ranks_match_the_single_process_oracle():
    import oracle as O
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in range(ws)), key=lambda r: r[0])
    for pr in procs:
        pr.join(timeout=120)
    assert all(pr.exitcode == 0 for pr in procs), [pr.exitcode for pr in procs]

    wl = _case()
    p = O.params_from(wl.params())
    T = O.taps(p)
    loc = O.locate(p, wl.u, wl.v, wl.w)
    want_grid = O.grid_separable(p, loc, wl.vis, wl.weight, T)
    want_pred = O.degrid_separable(p, loc, _model(wl.grid_size), wl.weight, T)
    want_img = O.wstack_image(p, wl.u, wl.v, wl.w, wl.vis, wl.weight, CENTRES)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))  # noqa: E731
    for rank, grid, pred, own, (lo, hi), image in res:
        # every rank holds the grid of all visibilities after the all-reduce
        assert rel(grid, want_grid) <= 1e-13, rank
        # predictions: the same arithmetic per visibility
        assert np.array_equal(pred, want_pred), rank
        assert np.array_equal(own, want_pred[lo:hi]), rank
        assert rel(image, want_img) <= 1e-12, rank
    # the shards split the visibilities
    assert res[0][4] == (0, res[1][4][0]) and res[1][4][1] == wl.nvis
