"""Integer arithmetic claims the GPU plan relies on, checked on the CPU against
IEEE double and exact integer arithmetic.  Each check restates the kernel's
algorithm in Python (the CUDA code is checked bit-exactly against the oracle
by the GPU tests); these pin the claims that make the algorithms exact:

- locate's integer path: floor(fl(y + N/2) OS + 1/2) taken from the bits of
  y = fl(u fov) equals the IEEE double result whenever y OS + 1/2 lies
  outside the fall-back margin N OS 2^-53 of an integer;
- floor(n / T) = (n ceil(2^32 / T)) >> 32 for 0 <= n < 2^26, 8 <= T <= 64;
- the sub-block-major sort key is a bijection onto 0 .. 32 ceil(T/4)^2 - 1.
"""
import math
import struct

import numpy as np
import pytest


def _fast_bounds(N, os_log2):
    half_span = (N << os_log2) // 2
    e = 0
    while e < 21 and (1 << (e + 1)) <= half_span:
        e += 1
    elim = e if (1 << e) <= half_span else -1
    near = ((N << os_log2) >> 13) + 2
    return elim, near


def _int_path(y, N, os_log2, elim, near):
    """('ok', t), ('fp64', None) or ('drop', None), as the kernel decides."""
    b = struct.unpack("<q", struct.pack("<d", y))[0]
    eb = (b >> 52) & 0x7FF
    if eb == 0x7FF:
        return "drop", None
    if eb == 0:
        z = (-1 if b < 0 else 0) + (1 << 39)
    else:
        ey = eb - 1023 + os_log2
        if ey >= elim:
            return "fp64", None
        m = (b & 0xFFFFFFFFFFFFF) | (1 << 52)
        sh = ey - 12
        if sh >= 0:
            a = m << sh
            a = -a if b < 0 else a
        elif sh > -53:
            q = m >> (-sh)
            rem = (m & ((1 << -sh) - 1)) != 0
            a = (-q - (1 if rem else 0)) if b < 0 else q
        else:
            a = -1 if b < 0 else 0
        z = a + (1 << 39)
    fr = z & ((1 << 40) - 1)
    if fr <= near or fr >= (1 << 40) - near:
        return "fp64", None
    return "ok", ((N // 2) << os_log2) + (z >> 40)


def _ieee_t(y, N, OS):
    x = y + float(N // 2)  # IEEE double add
    return math.floor(x * OS + 0.5)  # x OS exact; + 0.5 rounded, then floor


def _adversarial(N, OS, rng, n_rand=20000, n_ties=2000):
    H = N // 2
    ys = list(rng.uniform(-H - 5, H + 5, n_rand))
    ys += list(rng.uniform(-1, 1, 2000) * 10.0 ** rng.integers(-30, 3, 2000))
    for k in rng.integers(-H * OS, H * OS, n_ties):
        base = (float(k) - 0.5) / OS
        ys.append(base)
        up = dn = base
        for _ in range(3):
            up = float(np.nextafter(up, np.inf))
            dn = float(np.nextafter(dn, -np.inf))
            ys += [up, dn]
    for k in rng.integers(1, 1 << 40, n_ties):
        ys.append(float(k) * 2.0 ** (int(rng.integers(-20, 11)) - 40) - H)
    ys += [0.0, -0.0, 5e-324, -5e-324, float(H), -float(H), 0.5 / OS, -0.5 / OS,
           0.5 / OS - 2.0 ** -60, -0.5 / OS + 2.0 ** -60]
    return ys


@pytest.mark.parametrize("N,OS", [(4096, 16), (256, 8), (1000, 4), (96, 16), (8192, 256)])
def test_locate_integer_path_equals_ieee(N, OS):
    os_log2 = OS.bit_length() - 1
    elim, near = _fast_bounds(N, os_log2)
    rng = np.random.default_rng(N + OS)
    n_ok = 0
    for y in _adversarial(N, OS, rng):
        kind, t = _int_path(y, N, os_log2, elim, near)
        if kind == "ok":
            n_ok += 1
            assert t == _ieee_t(y, N, OS), (y, N, OS)
    assert n_ok > 10000  # the integer path is the common one


def test_locate_integer_path_falls_back_at_ties():
    """Values exactly on an oversample boundary (y OS + 1/2 an integer) and
    within a few ulps of it never take the integer path."""
    N, OS = 4096, 16
    elim, near = _fast_bounds(N, 4)
    for k in range(-100, 100):
        y = (k - 0.5) / OS
        for v in (y, float(np.nextafter(y, np.inf)), float(np.nextafter(y, -np.inf))):
            assert _int_path(v, N, 4, elim, near)[0] == "fp64"


@pytest.mark.parametrize("T", range(8, 65, 2))
def test_tile_division_by_multiply_high(T):
    M = (2 ** 32 + T - 1) // T
    for lo, hi in ((0, 1 << 16), ((1 << 26) - (1 << 16), 1 << 26)):
        n = np.arange(lo, hi, dtype=np.uint64)
        assert np.array_equal((n * np.uint64(M)) >> np.uint64(32), n // np.uint64(T))


@pytest.mark.parametrize("T", [8, 16, 30, 32, 48, 56, 62, 64])
def test_sub_block_sort_key_is_a_bijection(T):
    M = (2 ** 32 + T - 1) // T
    div = lambda n: (n * M) >> 32  # noqa: E731
    E = (T + 3) // 4
    seen = set()
    for ly in range(T):
        for lx in range(T):
            for cj in (0, 1):
                sx, sy = div(lx * 4), div(ly * 4)
                x0, y0 = (sx * T + 3) >> 2, (sy * T + 3) >> 2
                assert 0 <= lx - x0 < E and 0 <= ly - y0 < E
                k = ((((sx * 4 + sy) << 1) | cj) * E + (ly - y0)) * E + (lx - x0)
                assert 0 <= k < 32 * E * E <= 8192 and k not in seen
                seen.add(k)
