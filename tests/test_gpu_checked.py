"""The bounds-checked build (libsepw_checked.so, -DSEPW_CHECKED=1).

On valid input it must give the default build's results (tiled gridding and
degridding against the FP64 oracle, status OK).  With one plan slot
corrupted through the checked build's test hook (its visibility index out of
range, or its record's w-plane beyond the table), the register-block tiled
kernels must catch it before any access: status SEPW_EBOUNDS, the slot's
visibility skipped by both kernels, everything else as the oracle computes
it without that visibility.  The skipped visibility is found as the one
prediction the degridder left at its sentinel value.  The corrupting hook is
refused by the default build, which has no such checks.

The checked library is chosen when the binding is imported, so the checked
runs happen in a child process."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import torch
import oracle as O
import synth
import paper_1511_07152_gb300.sepw as S
assert S.sepw_checked_build()
res = {}
for name, S_, seed in (("S16", 16, 21), ("S8", 8, 22)):
    wl = synth.random_case(seed, 6000, 160, S_, 16, 17, edge_fraction=0.1)
    p = O.params_from(wl.params())
    loc = O.locate(p, wl.u, wl.v, wl.w)
    T = O.taps(p)
    rng = np.random.default_rng(seed)
    N = wl.grid_size
    X = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex64)
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TILED))
    taps = S.sepw_make_taps(ctx)
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w", "vis", "weight")}
    Xd = torch.from_numpy(X).cuda()
    for case, which, value in (("clean", None, 0), ("perm", 0, wl.nvis + 100),
                               ("plane", 1, p.P + 3)):
        S.sepw_plan(ctx, d["u"], d["v"], d["w"])  # a fresh plan for each case
        if which is not None:
            S.sepw_test_corrupt_plan(ctx, which, 7, value)
        g = torch.zeros((N, N), dtype=torch.complex64, device="cuda")
        S.sepw_grid_planned(ctx, taps, d["vis"], d["weight"], g)
        out = torch.full((wl.nvis,), complex(7, 7), dtype=torch.complex64, device="cuda")
        S.sepw_degrid_planned(ctx, taps, Xd, d["weight"], out)
        status = S.sepw_device_status(ctx)
        got_g = g.cpu().numpy()
        got_p = out.cpu().numpy()
        skipped = np.flatnonzero(got_p == np.complex64(complex(7, 7)))
        keep = loc["keep"].copy()
        keep[skipped] = False
        loc2 = dict(loc)
        loc2["keep"] = keep
        want_g = O.grid_separable(p, loc2, wl.vis, wl.weight, T)
        want_p = O.degrid_separable(p, loc2, X, wl.weight, T)
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        mask = np.ones(wl.nvis, bool)
        mask[skipped] = False
        res[name + "_" + case] = dict(status=int(status), skipped=[int(k) for k in skipped],
                                      dropped_by_locate=[int(k) for k in skipped
                                                         if not loc["keep"][k]],
                                      grid_err=rel(got_g, want_g),
                                      pred_err=rel(got_p[mask], want_p[mask]))
    ctx.close()
print(json.dumps(res))
"""


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_07152_gb300 import build
    build.build()
    build.build(checked=True)
    import paper_1511_07152_gb300.sepw as S
    return torch, S


def test_default_build_refuses_the_corrupting_hook(env):
    torch, S = env
    assert not S.sepw_checked_build()
    import synth
    wl = synth.random_case(21, 600, 160, 16, 16, 17)
    ctx = S.sepw_create(S.make_params(**wl.params(), form=S.FORM_TILED))
    d = {k: torch.from_numpy(getattr(wl, k)).cuda() for k in ("u", "v", "w")}
    S.sepw_plan(ctx, d["u"], d["v"], d["w"])
    with pytest.raises(S.SepwError) as e:
        S.sepw_test_corrupt_plan(ctx, 0, 7, 10 ** 6)
    assert e.value.status == S.ENOTSUP
    ctx.close()


def test_checked_build_catches_corrupt_plan_slots(env):
    env_vars = dict(os.environ, SEPW_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env_vars,
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for name in ("S16", "S8"):
        clean = res[name + "_clean"]
        assert clean["status"] == 0, clean
        assert clean["skipped"] == []
        assert clean["grid_err"] <= 1e-5 and clean["pred_err"] <= 1e-5, clean
        for case in ("perm", "plane"):
            c = res[f"{name}_{case}"]
            assert c["status"] == -8, c  # SEPW_EBOUNDS
            # exactly one visibility skipped, and one that locate had kept
            assert len(c["skipped"]) == 1 and c["dropped_by_locate"] == [], c
            assert c["grid_err"] <= 1e-5 and c["pred_err"] <= 1e-5, c
