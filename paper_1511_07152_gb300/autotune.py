"""Autotuner for the tiled and tensor-core forms: form, tile edge T and the
visibility-per-tile schedule.

For a given geometry (grid size, support, oversampling, planes) and a
representative set of visibilities, every candidate (form, T) is timed on the
GPU through the C ABI (plan + grid, CUDA events, median of a few runs) and the
fastest one that meets the caller's accuracy class is kept; then, for that
(form, T), the schedule of the plan (visibilities per work item, and for the
FP32 block gridder the parts of an item a warp takes at a time) is tuned the
same way.  Results are cached in a JSON file keyed by the GPU name and the
geometry, so a pipeline tunes once and reuses the choice.

Host logic (candidate lists, keys, the choice, the cache) is plain Python and
is tested without a GPU; timing needs the CUDA library.
"""
from __future__ import annotations

import json
import os
import statistics
from dataclasses import dataclass, field

FORM_NAMES = {0: "plain", 1: "tiled", 2: "tc_bf16", 3: "tc_fp16", 4: "tc_fp16x2",
              5: "tc_bf16x2", 6: "tc_tf32"}
# accuracy class of each form: the grid's relative L2 error bound it meets
FORM_ERROR = {"plain": 1e-5, "tiled": 1e-5, "tc_bf16": 1e-2, "tc_fp16": 1.5e-3,
              "tc_fp16x2": 1e-5, "tc_bf16x2": 1e-5, "tc_tf32": 1.5e-3}


def candidate_tiles(support: int, form: str) -> list[int]:
    """Even tile edges T worth timing: T + S - 1 <= 64 (the tiled forms'
    shared-memory window) or <= 32 (the tensor-core gridder's window, S <= 16
    only).  The plain form has no tiles (one candidate, 0)."""
    if form == "plain":
        return [0]
    if form.startswith("tc"):
        if support > 16:
            return []
        tmax = (33 - support) & ~1
        return [T for T in (tmax - 8, tmax - 4, tmax) if T >= 8]
    return [T for T in (16, 24, 32, 40, 48, 56) if T + support - 1 <= 64]


def candidate_schedules(form: str) -> list[tuple[int, int]]:
    """(chunk, grid_parts) candidates for a form: work items of 512 .. 2048
    visibilities; the FP32 tiled form also tries whole items (1) and eighths
    (8) per warp unit besides the density rule (0).  The plain form has no
    plan schedule."""
    if form == "plain":
        return [(0, 0)]
    chunks = (512, 1024, 2048)
    parts = (0, 1, 8) if form == "tiled" else (0,)
    return [(c, q) for c in chunks for q in parts]


def cache_key(gpu: str, grid_size: int, support: int, oversample: int, n_wplanes: int,
              batched: bool) -> str:
    return f"{gpu}|N{grid_size}|S{support}|OS{oversample}|P{n_wplanes}|b{int(batched)}"


def choose(timings: dict, max_error: float) -> tuple[str, int, float]:
    """Fastest (form, T) whose accuracy class meets max_error.
    timings: {(form, T): [ms, ...]}."""
    best = None
    for (form, T), ms in timings.items():
        if FORM_ERROR[form] > max_error or not ms:
            continue
        m = statistics.median(ms)
        if best is None or m < best[2]:
            best = (form, T, m)
    if best is None:
        raise ValueError("no candidate meets the accuracy bound")
    return best


@dataclass
class TuneCache:
    path: str
    data: dict = field(default_factory=dict)

    @classmethod
    def load(cls, path: str) -> "TuneCache":
        try:
            with open(path) as f:
                return cls(path, json.load(f))
        except (OSError, ValueError):
            return cls(path, {})

    def get(self, key: str):
        return self.data.get(key)

    def put(self, key: str, value: dict):
        self.data[key] = value
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def default_cache_path() -> str:
    return os.environ.get("SEPW_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "sepw_tune.json"))


def tune(params: dict, u, v, w, vis, weight, max_error: float = 1e-5, forms=None,
         vis_offsets=None, reps: int = 3, cache_path: str | None = None, use_cache=True):
    """Pick the form and tile for this geometry.  params: grid_size, fov,
    support, oversample, n_wplanes, w_max[, gamma, kb_beta].  u, v, w, vis,
    weight: CUDA tensors of a representative sample.  vis_offsets: batched
    layout (host array) or None.  Returns dict(form=..., tile=..., ms=...,
    timings=...)."""
    import torch

    from . import sepw as S

    gpu = torch.cuda.get_device_name()
    key = cache_key(gpu, params["grid_size"], params["support"], params["oversample"],
                    params["n_wplanes"], vis_offsets is not None)
    cache = TuneCache.load(cache_path or default_cache_path())
    if use_cache:
        hit = cache.get(key)
        if hit and FORM_ERROR[hit["form"]] <= max_error:
            return hit
    forms = forms or [f for f in ("plain", "tiled", "tc_fp16x2", "tc_bf16x2", "tc_tf32", "tc_fp16",
                                  "tc_bf16") if FORM_ERROR[f] <= max_error]
    codes = {v_: k for k, v_ in FORM_NAMES.items()}
    N = params["grid_size"]
    ng = 1 if vis_offsets is None else len(vis_offsets) - 1
    grid = torch.zeros((ng, N, N), dtype=torch.complex64, device="cuda")
    timings = {}
    stream = torch.cuda.current_stream()
    for form in forms:
        for T in candidate_tiles(params["support"], form):
            ctx = S.sepw_create(S.make_params(**params, tile=T, form=codes[form]))
            taps = S.sepw_make_taps(ctx)
            ms = []
            for r in range(reps + 1):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                if vis_offsets is None:
                    S.sepw_plan(ctx, u, v, w)
                else:
                    S.sepw_plan_batched(ctx, vis_offsets, u, v, w)
                S.sepw_grid_planned(ctx, taps, vis, weight, grid)
                b.record(stream)
                torch.cuda.synchronize()
                if r > 0:  # first run warms up
                    ms.append(a.elapsed_time(b))
            timings[(form, T)] = ms
            ctx.close()
    form, T, m = choose(timings, max_error)
    # the schedule of the chosen (form, T)
    sched = {}
    ctx = S.sepw_create(S.make_params(**params, tile=T, form=codes[form]))
    taps = S.sepw_make_taps(ctx)
    for chunk, parts in candidate_schedules(form):
        if form != "plain":
            S.sepw_set_schedule(ctx, chunk, parts)
        ms = []
        for r in range(reps + 1):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if vis_offsets is None:
                S.sepw_plan(ctx, u, v, w)
            else:
                S.sepw_plan_batched(ctx, vis_offsets, u, v, w)
            S.sepw_grid_planned(ctx, taps, vis, weight, grid)
            b.record(stream)
            torch.cuda.synchronize()
            if r > 0:
                ms.append(a.elapsed_time(b))
        sched[(chunk, parts)] = statistics.median(ms)
    ctx.close()
    (chunk, parts), m2 = min(sched.items(), key=lambda kv: kv[1])
    out = dict(form=form, tile=T, chunk=chunk, grid_parts=parts, ms=min(m, m2),
               timings={f"{k[0]}:T{k[1]}": statistics.median(v_) for k, v_ in timings.items()},
               schedule_timings={f"chunk{k[0]}:parts{k[1]}": v_ for k, v_ in sched.items()})
    cache.put(key, out)
    return out
