"""Host logic of the autotuner (no GPU)."""
import json

import pytest

from paper_1511_07152_gb300 import autotune as A


def test_candidate_tiles_respect_window():
    for S in (2, 8, 12, 16, 32):
        ts = A.candidate_tiles(S, "tiled")
        assert ts and all(T % 2 == 0 and T + S - 1 <= 64 for T in ts)
    for S in (2, 8, 12, 16):
        ts = A.candidate_tiles(S, "tc_bf16")
        assert ts and all(T % 2 == 0 and 8 <= T and T + S - 1 <= 32 for T in ts)
    assert A.candidate_tiles(32, "tc_bf16") == []  # tensor-core forms take S <= 16
    assert A.candidate_tiles(16, "tc_fp16") == [8, 12, 16]
    assert A.candidate_tiles(12, "tc_bf16x2") == [12, 16, 20]


def test_choose_respects_accuracy_class():
    timings = {("tiled", 32): [3.0, 3.1, 2.9], ("tc_bf16", 48): [1.0, 1.0],
               ("tc_fp16", 48): [1.2, 1.3], ("tiled", 16): [4.0]}
    assert A.choose(timings, 1e-5)[:2] == ("tiled", 32)
    assert A.choose(timings, 2e-3)[:2] == ("tc_fp16", 48)
    assert A.choose(timings, 1e-2)[:2] == ("tc_bf16", 48)
    with pytest.raises(ValueError):
        A.choose({("tc_bf16", 48): [1.0]}, 1e-5)


def test_cache_roundtrip(tmp_path):
    p = tmp_path / "sub" / "tune.json"
    c = A.TuneCache.load(str(p))
    key = A.cache_key("GB300", 4096, 16, 16, 128, False)
    assert c.get(key) is None
    c.put(key, {"form": "tiled", "tile": 32, "ms": 3.0})
    c2 = A.TuneCache.load(str(p))
    assert c2.get(key)["tile"] == 32
    assert json.load(open(p))[key]["form"] == "tiled"
    assert key != A.cache_key("GB300", 4096, 16, 16, 128, True)


def test_candidate_schedules():
    assert A.candidate_schedules("plain") == [(0, 0)]
    tiled = A.candidate_schedules("tiled")
    assert (2048, 0) in tiled and (512, 8) in tiled and len(tiled) == 9
    tc = A.candidate_schedules("tc_bf16x2")
    assert all(q == 0 for _, q in tc) and {c for c, _ in tc} == {512, 1024, 2048}
    for c, q in tiled + tc:
        assert 64 <= c <= 2048 and c % 32 == 0 and 0 <= q <= 16
