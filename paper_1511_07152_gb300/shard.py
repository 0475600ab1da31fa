"""Visibility-sharded gridding, degridding and W-stacking imaging over ranks
(one process and one GPU per rank, torch.distributed).

Gridding is linear in the visibilities (Sec. 5: every visibility adds its own
separable update to the grid), and so is the hybrid W-stacking image (Sec. 4.3:
each slice's grid, imaged and phase-corrected, then summed).  So the
visibilities split into contiguous shards, one per rank, and:
  - gridding: each rank grids its shard into a private N x N grid, then one
    all-reduce (sum) of the grid gives every rank the grid of all
    visibilities;
  - degridding (prediction): the model grid is broadcast from one rank, each
    rank predicts its own shard, no reduction; the predictions can be
    gathered in the global order;
  - W stacking: each rank images its shard through every slice, then one
    all-reduce (sum) of the N x N image.
The per-shard work is a function argument: `cuda_grid_fn` and friends bind it
to a context of the CUDA library (the production path; there is no CPU
fallback), and any other function with the same signature can stand in (the
CPU tests use the FP64 oracle on gloo ranks).  Collectives run on the default
process group unless `group` is given; complex tensors travel as their real
views, so NCCL and gloo both apply.
"""
from __future__ import annotations


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous shard [lo, hi) of n items for `rank` of `world`; shard sizes
    differ by at most one and concatenate in rank order to 0 .. n."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n >= 0")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def _rank_world(group):
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def _real(t):
    import torch
    return torch.view_as_real(t) if t.is_complex() else t


def allreduce_sum(t, group=None):
    """In-place sum of t over the ranks (a no-op for one rank)."""
    import torch.distributed as dist
    _, world = _rank_world(group)
    if world > 1:
        dist.all_reduce(_real(t), op=dist.ReduceOp.SUM, group=group)
    return t


def grid_sharded(grid_shard_fn, u, v, w, vis, weight, grid, group=None):
    """Grid this rank's shard (u, v, w, vis, weight: the shard's arrays; weight
    may be None) into `grid` (accumulated, +=), then sum the grid over the
    ranks.  grid_shard_fn(u, v, w, vis, weight, grid) grids one shard."""
    grid_shard_fn(u, v, w, vis, weight, grid)
    return allreduce_sum(grid, group)


def degrid_sharded(degrid_shard_fn, u, v, w, model_grid, weight, src: int = 0,
                   gather: bool = False, n_total: int | None = None, group=None):
    """Predict this rank's shard from the model grid of rank `src` (broadcast
    to every rank first, in place).  degrid_shard_fn(u, v, w, grid, weight)
    returns the shard's predictions.  With gather=True every rank receives
    all predictions in the global order (shards contiguous in rank order,
    n_total visibilities in all); otherwise the shard's own."""
    import torch
    import torch.distributed as dist
    rank, world = _rank_world(group)
    if world > 1:
        dist.broadcast(_real(model_grid), src=src, group=group)
    out = degrid_shard_fn(u, v, w, model_grid, weight)
    if not gather or world == 1:
        return out
    if n_total is None:
        raise ValueError("gather needs n_total")
    sizes = [shard_bounds(n_total, r, world) for r in range(world)]
    m = max(hi - lo for lo, hi in sizes)
    pad = torch.zeros((m,), dtype=out.dtype, device=out.device)
    pad[: out.numel()] = out
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather([_real(p) for p in parts], _real(pad), group=group)
    return torch.cat([parts[r][: hi - lo] for r, (lo, hi) in enumerate(sizes)])


def wstack_image_sharded(image_shard_fn, u, v, w, vis, weight, image, group=None):
    """Hybrid W-stacking image of all ranks' visibilities: each rank images
    its shard through every slice (image_shard_fn(u, v, w, vis, weight,
    image) overwrites `image` with the shard's image), then one all-reduce
    (sum) of the image."""
    image_shard_fn(u, v, w, vis, weight, image)
    return allreduce_sum(image, group)


# ---- per-shard functions on the CUDA library --------------------------------


def cuda_grid_fn(ctx, taps):
    """Per-shard gridding through the C ABI (sepw_grid) of a context."""
    from . import sepw as S

    def f(u, v, w, vis, weight, grid):
        S.sepw_grid(ctx, taps, u, v, w, vis, weight, grid)
    return f


def cuda_degrid_fn(ctx, taps):
    """Per-shard prediction through the C ABI (sepw_degrid) of a context."""
    import torch

    from . import sepw as S

    def f(u, v, w, grid, weight):
        out = torch.empty(u.numel(), dtype=torch.complex64, device=u.device)
        S.sepw_degrid(ctx, taps, u, v, w, grid, weight, out)
        return out
    return f


def cuda_wstack_image_fn(ctx, taps, centres):
    """Per-shard hybrid W-stacking image through the C ABI (sepw_wstack_plan,
    sepw_grid_planned, sepw_wstack_image) of a context."""
    import torch

    from . import sepw as S

    def f(u, v, w, vis, weight, image):
        N = ctx.params.grid_size
        S.sepw_wstack_plan(ctx, centres, u, v, w)
        grids = torch.zeros((len(centres), N, N), dtype=torch.complex64, device=u.device)
        S.sepw_grid_planned(ctx, taps, vis, weight, grids)
        S.sepw_wstack_image(ctx, grids, image)
    return f
