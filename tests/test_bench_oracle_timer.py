"""The bench's CPU baseline runs the FP64 oracle on every host core by
splitting the visibilities over threads and summing their grids: the summed
grid must be the oracle's grid of all visibilities (rounding order aside)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_threaded_oracle_sums_to_the_single_thread_grid():
    import bench
    import oracle as O
    import synth
    wl = synth.random_case(71, 5000, 128, 8, 8, 9, edge_fraction=0.1)
    t = bench.OracleTimer(wl, wl.nvis, threads=3)
    try:
        dt = t.step()
    finally:
        t.close()
    assert dt > 0 and t.nt == 3
    p = O.params_from(t.sub.params())
    loc = O.locate(p, t.sub.u, t.sub.v, t.sub.w)
    want = O.grid_separable(p, loc, t.sub.vis, t.sub.weight, O.taps(p))
    assert np.linalg.norm(t.total - want) <= 1e-13 * np.linalg.norm(want)
    # the shards cover every visibility once
    assert t.bounds[0][0] == 0 and t.bounds[-1][1] == t.sub.nvis
