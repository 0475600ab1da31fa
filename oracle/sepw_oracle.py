"""FP64 oracle for separable W-projection gridding (Merry 2015).

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg use this module.  Plain numpy (float64 / complex128) plus the
plain-C loops of ``sepw_oracle.c``.  Library primitives used as steps: a
matrix product (DFT sums), ``numpy.fft`` (pinned against the direct DFT), and
``numpy.i0``.

Geometry and notation (Sec. 2):
  * u, v, w in wavelengths; l, m direction cosines, n = sqrt(1 - l^2 - m^2).
  * Grid N x N, row-major [v][u]; cell size du = 1 / fov; the u = 0 column is
    N/2.  Image pixel a has l_a = nu_a * fov with nu_a = (a - N/2) / N (the
    image fraction, cycles per grid cell).
  * Taper c1 (the antialiasing kernel's inverse transform, Sec. 2): the
    Kaiser-Bessel window C(x) = I0(beta sqrt(1 - (2x/S)^2)), |x| <= S/2 cells,
    has the closed-form transform S sinh(z)/z, z = sqrt(beta^2 - (pi S nu)^2)
    (sin form when the root is imaginary); c1 is that, normalised to c1(0)=1.

Readings where the paper is silent are stated in the docstring of the
function that takes them.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import numpy as np

from . import build_oracle

# --------------------------------------------------------------------------
# parameters
# --------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Params:
    grid_size: int
    fov: float
    support: int
    oversample: int
    n_wplanes: int
    w_max: float
    gamma: float = 5.0 / 24.0
    kb_beta: float | None = None

    def __post_init__(self):
        if self.kb_beta is None:
            object.__setattr__(self, "kb_beta", 2.34 * self.support)
        if self.grid_size % 2 or self.support % 2:
            raise ValueError("grid_size and support must be even")

    @property
    def N(self):
        return self.grid_size

    @property
    def S(self):
        return self.support

    @property
    def OS(self):
        return self.oversample

    @property
    def P(self):
        return self.n_wplanes


def params_from(d: dict) -> Params:
    return Params(**{k: d[k] for k in ("grid_size", "fov", "support", "oversample",
                                       "n_wplanes", "w_max", "gamma", "kb_beta")})


# --------------------------------------------------------------------------
# pixel geometry, taper, phase screens (Secs. 2-3)
# --------------------------------------------------------------------------


def pixel_nu(N: int) -> np.ndarray:
    """Image fraction nu_a = (a - N/2)/N of pixel a (cycles per grid cell)."""
    return (np.arange(N, dtype=np.float64) - N // 2) / N


def pixel_l(N: int, fov: float) -> np.ndarray:
    """Direction cosine of pixel a: l_a = nu_a * fov (du = 1/fov)."""
    return pixel_nu(N) * fov


def kb_kernel(x, S: int, beta: float):
    """Kaiser-Bessel uv-domain window C(x) = I0(beta sqrt(1-(2x/S)^2)),
    |x| <= S/2 cells, zero outside (the antialiasing kernel C of Sec. 2)."""
    x = np.asarray(x, np.float64)
    r = 1.0 - (2.0 * x / S) ** 2
    out = np.zeros_like(x)
    ok = r >= 0
    out[ok] = np.i0(beta * np.sqrt(r[ok]))
    return out


def kb_taper(nu, S: int, beta: float):
    """c1(nu): continuous Fourier transform of kb_kernel, S sinh(z)/z with
    z = sqrt(beta^2 - (pi S nu)^2), normalised so c1(0) = 1.  Evaluated as
    (beta/z) e^(z-beta) (1-e^(-2z)) / (1-e^(-2 beta)) to avoid overflow."""
    nu = np.asarray(nu, np.float64)
    z2 = beta * beta - (np.pi * S * nu) ** 2
    out = np.empty_like(nu)
    den = 1.0 - math.exp(-2.0 * beta)
    pos = z2 > 0
    z = np.sqrt(z2[pos])
    out[pos] = (beta / z) * np.exp(z - beta) * (-np.expm1(-2.0 * z)) / den
    neg = z2 < 0
    z = np.sqrt(-z2[neg])
    out[neg] = (beta / z) * np.sin(z) * 2.0 * math.exp(-beta) / den
    zero = z2 == 0
    out[zero] = beta * 2.0 * math.exp(-beta) / den
    return out


def n_minus_1(l, m):
    """n - 1 with n = sqrt(1 - l^2 - m^2), written without cancellation."""
    r2 = l * l + m * m
    return -r2 / (1.0 + np.sqrt(1.0 - r2))


def g_exact(w, l, m):
    """g_w(l, m) = exp(2 pi i w (n - 1)) (Sec. 2)."""
    return np.exp(2j * np.pi * w * n_minus_1(l, m))


def g1(w, l, gamma):
    """1-D screen g1_w(l) = exp(2 pi i w (-l^2/2 - gamma l^4)) (Eq. gt)."""
    return np.exp(2j * np.pi * w * (-0.5 * l * l - gamma * l ** 4))


def g_separable(w, l, m, gamma):
    """Separable screen g~_w(l, m) = g1_w(l) g1_w(m) (Eq. gt)."""
    return g1(w, l, gamma) * g1(w, m, gamma)


def plane_w(P: int, w_max: float) -> np.ndarray:
    """w of plane p: p * w_max / (P - 1), p = 0..P-1, over |w| in [0, w_max]
    (reading: planes cover |w|; w < 0 uses the conjugate kernel)."""
    if P == 1:
        return np.zeros(1)
    return np.arange(P, dtype=np.float64) * w_max / (P - 1)


# --------------------------------------------------------------------------
# kernels: 1-D taps (Eq. gt) and the exact 2-D table (Sec. 2)
# --------------------------------------------------------------------------


def tap_offsets(S: int, OS: int) -> np.ndarray:
    """d[o][j] = j - S/2 + 1 - o/OS: offset (cells) of footprint column j
    from a visibility at oversampled position c + o/OS."""
    j = np.arange(S, dtype=np.float64)
    o = np.arange(OS, dtype=np.float64)
    return (j[None, :] - S / 2 + 1) - o[:, None] / OS


def _dft_rows(S: int, OS: int, N: int) -> np.ndarray:
    """E[(o, j), a] = exp(-2 pi i d[o][j] nu_a)."""
    d = tap_offsets(S, OS).reshape(-1)
    return np.exp(-2j * np.pi * d[:, None] * pixel_nu(N)[None, :])


def taps(p: Params, planes=None) -> np.ndarray:
    """1-D GCF table T[p][o][j] = F1_{w_p}(j - S/2 + 1 - o/OS), complex128.

    F1_w is the transform of c1 g1_w (Sec. 2: the GCF is the transform of the
    product of the screen and the taper; Eq. gt gives the separable screen),
    taken as the DFT over the N image pixels that the grid's FFT produces:
        F1_w(d) = (1/N) sum_a c1(nu_a) g1_w(l_a) exp(-2 pi i d nu_a).
    With full support this makes gridding + unnormalised inverse DFT + division
    by c1 reproduce the direct sum exactly (pinned by the tests)."""
    N, S, OS = p.N, p.S, p.OS
    wp = plane_w(p.P, p.w_max)
    if planes is not None:
        wp = wp[np.asarray(planes)]
    nu = pixel_nu(N)
    l = nu * p.fov
    h = kb_taper(nu, S, p.kb_beta)[None, :] * g1(wp[:, None], l[None, :], p.gamma)
    E = _dft_rows(S, OS, N)
    T = (h @ E.T) / N
    return T.reshape(len(wp), OS, S)


def exact_table(p: Params, planes=None, screen: str = "exact") -> np.ndarray:
    """Full 2-D GCF table K[p][ov][ou][k][j] = F_w(d_u, d_v) with
    F_w(d_u, d_v) = (1/N^2) sum_{a,b} c1(nu_a) c1(nu_b) g(l_a, m_b)
                     exp(-2 pi i (d_u nu_a + d_v nu_b)),
    g = g_w (screen='exact', the non-separable kernel the paper replaces) or
    g~_w (screen='separable', for the outer-product pin).  Small N only."""
    N, S, OS = p.N, p.S, p.OS
    wp = plane_w(p.P, p.w_max)
    if planes is not None:
        wp = wp[np.asarray(planes)]
    nu = pixel_nu(N)
    l = nu * p.fov
    c = kb_taper(nu, S, p.kb_beta)
    L, M = np.meshgrid(l, l)  # [b][a]: L = l_a, M = m_b
    E = _dft_rows(S, OS, N)
    out = np.empty((len(wp), OS, OS, S, S), np.complex128)
    for i, w in enumerate(wp):
        g = g_exact(w, L, M) if screen == "exact" else g_separable(w, L, M, p.gamma)
        H = c[:, None] * c[None, :] * g  # [b][a]
        K = (E @ H @ E.T) / (N * N)      # [(ov,k), (ou,j)]
        out[i] = K.reshape(OS, S, OS, S).transpose(0, 2, 1, 3)
    return out


# --------------------------------------------------------------------------
# locating a visibility on the grid and in the plane stack
# --------------------------------------------------------------------------


def locate(p: Params, u, v, w, wrap: bool = False) -> dict:
    """Cell, oversample offset, plane and conjugation of each visibility.

    Readings (the paper fixes none of these; IEEE double, each operation
    rounded separately, no fused multiply-add):
      x = u*fov + N/2;  t = floor(x*OS + 0.5)  (ties toward +inf)
      c = floor(t / OS);  o = t - c*OS
      the footprint c - S/2 + 1 .. c + S/2 must lie in [0, N), else drop;
      r = (P - 1)/w_max;  plane = floor(|w|*r + 0.5), drop if > P - 1;
      conj = (w < 0): the kernel for -w is the conjugate of the kernel for |w|.
    Non-finite coordinates are dropped.  wrap=True skips the footprint test
    (cells are then taken modulo N by the gridder; used only by the pins that
    compare full-support gridding with the direct sums)."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    w = np.asarray(w, np.float64)
    N, S, OS, P = p.N, p.S, p.OS, p.P
    half = float(N // 2)

    def axis(coord):
        with np.errstate(invalid="ignore", over="ignore"):
            x = coord * p.fov + half
            t = np.floor(x * float(OS) + 0.5)
            ok = np.isfinite(t) & (np.abs(t) < 2.0 ** 40)
        ti = np.where(ok, t, 0.0).astype(np.int64)
        c = np.floor_divide(ti, OS)
        o = ti - c * OS
        f = c - (S // 2) + 1
        if not wrap:
            ok &= (f >= 0) & (f + S - 1 <= N - 1)
        return c, o, ok

    cu, ou, oku = axis(u)
    cv, ov, okv = axis(v)
    r = (P - 1) / p.w_max if P > 1 else 0.0
    with np.errstate(invalid="ignore", over="ignore"):
        pf = np.floor(np.abs(w) * r + 0.5)
        okw = np.isfinite(w) & np.isfinite(pf) & (pf <= P - 1)
    plane = np.where(okw, pf, 0.0).astype(np.int64)
    keep = oku & okv & okw
    z = lambda a: np.where(keep, a, 0)  # noqa: E731
    return dict(cu=z(cu).astype(np.int32), cv=z(cv).astype(np.int32),
                ou=z(ou).astype(np.int32), ov=z(ov).astype(np.int32),
                plane=z(plane).astype(np.int32), conj=(w < 0) & keep,
                keep=keep)


# --------------------------------------------------------------------------
# plain-C loops
# --------------------------------------------------------------------------

_LIB = None
_I32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_U8 = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_F64 = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def _clib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_oracle.build())
        common = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                  _I32, _I32, _I32, _I32, _I32, _U8, _U8]
        lib.oracle_grid_separable.argtypes = common + [_F64, ctypes.c_void_p, _F64,
                                                       ctypes.c_void_p, ctypes.c_int32, _F64]
        lib.oracle_degrid_separable.argtypes = common + [_F64, ctypes.c_void_p, _F64,
                                                         ctypes.c_void_p, ctypes.c_int32, _F64]
        lib.oracle_grid_exact2d.argtypes = common + [_F64, ctypes.c_void_p, _F64,
                                                     ctypes.c_int32, _F64]
        rcommon = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                   ctypes.c_int32, ctypes.c_int32, _I32, _I32, _I32, _I32, _I32, _U8, _U8]
        lib.oracle_grid_residual.argtypes = rcommon + [_F64, ctypes.c_void_p, _F64, _F64]
        lib.oracle_degrid_residual.argtypes = rcommon + [_F64, ctypes.c_void_p, _F64, _F64]
        for f in (lib.oracle_grid_separable, lib.oracle_degrid_separable,
                  lib.oracle_grid_exact2d, lib.oracle_grid_residual,
                  lib.oracle_degrid_residual):
            f.restype = None
        _LIB = lib
    return _LIB


def _loc_args(loc):
    c = lambda a, t: np.ascontiguousarray(a, t)  # noqa: E731
    return (c(loc["cu"], np.int32), c(loc["cv"], np.int32), c(loc["ou"], np.int32),
            c(loc["ov"], np.int32), c(loc["plane"], np.int32),
            c(loc["conj"], np.uint8), c(loc["keep"], np.uint8))


def _c128(a):
    return np.ascontiguousarray(a, np.complex128).view(np.float64)


def _weight_arg(weight, n):
    if weight is None:
        return None, None
    wt = np.ascontiguousarray(weight, np.float64)
    assert wt.shape == (n,)
    return wt, wt.ctypes.data


def _tv_arg(Tv):
    if Tv is None:
        return None, None
    tv = _c128(Tv).reshape(-1)
    return tv, tv.ctypes.data


def grid_separable(p: Params, loc: dict, vis, weight, T, wrap=False, grid=None, Tv=None):
    """Separable gridder (Sec. 5), FP64: returns the N x N complex128 grid.
    Tv: separate v-direction table (facet screens, Sec. 4.1), default T."""
    n = len(loc["keep"])
    if p.S > 1024:
        raise ValueError("support > 1024")
    if grid is None:
        grid = np.zeros((p.N, p.N), np.complex128)
    visd = _c128(vis)
    wt, wptr = _weight_arg(weight, n)
    tv, tvptr = _tv_arg(Tv)
    gflat = grid.view(np.float64).reshape(-1)
    _clib().oracle_grid_separable(n, p.N, p.S, p.OS, *_loc_args(loc), visd, wptr,
                                  _c128(T).reshape(-1), tvptr, int(wrap), gflat)
    return grid


def degrid_separable(p: Params, loc: dict, grid, weight, T, wrap=False, Tv=None):
    """Separable degridder (the adjoint of grid_separable), FP64."""
    n = len(loc["keep"])
    out = np.zeros(n, np.complex128)
    wt, wptr = _weight_arg(weight, n)
    tv, tvptr = _tv_arg(Tv)
    _clib().oracle_degrid_separable(n, p.N, p.S, p.OS, *_loc_args(loc),
                                    _c128(grid).reshape(-1), wptr,
                                    _c128(T).reshape(-1), tvptr, int(wrap),
                                    out.view(np.float64))
    return out


def grid_exact2d(p: Params, loc: dict, vis, weight, K, wrap=False):
    """Exact 2-D-kernel W-projection gridder (Sec. 2), FP64."""
    n = len(loc["keep"])
    grid = np.zeros((p.N, p.N), np.complex128)
    wt, wptr = _weight_arg(weight, n)
    _clib().oracle_grid_exact2d(n, p.N, p.S, p.OS, *_loc_args(loc), _c128(vis), wptr,
                                _c128(K).reshape(-1), int(wrap),
                                grid.view(np.float64).reshape(-1))
    return grid


def residual_table(p: Params, Sr: int = None, OSr: int = None, K=None, T=None):
    """Stored correction of the separable kernel (Sec. 7: store and apply
    F_w - F~_w in a small full-dimension table):
        R[p][ov][ou][k][j] = F_w(d_u, d_v) - F1_w(d_u) F1_w(d_v)
    with F_w the exact 2-D kernel of exact_table and F1 the taps, on the Sr x Sr
    central footprint cells (first at k0 = (S - Sr)/2) and every
    (OS / OSr)-th oversample offset per axis.

    Reading (the paper leaves the table's support and sampling open): the
    truncated table keeps the central cells, and a visibility at fine offset o
    uses the coarse entry floor(o / (OS / OSr)).  Sr = S, OSr = OS gives the
    exact kernel back when added to the separable one."""
    S, OS = p.S, p.OS
    Sr = S if Sr is None else Sr
    OSr = OS if OSr is None else OSr
    if Sr < 1 or Sr > S or (S - Sr) % 2 or OSr < 1 or OS % OSr:
        raise ValueError("need 1 <= Sr <= S, S - Sr even, OSr dividing OS")
    K = exact_table(p) if K is None else K
    T = taps(p) if T is None else T
    full = K - T[:, :, None, :, None] * T[:, None, :, None, :]
    step, k0 = OS // OSr, (S - Sr) // 2
    return np.ascontiguousarray(full[:, ::step, ::step, k0:k0 + Sr, k0:k0 + Sr])


def _res_dims(p: Params, R):
    return int(R.shape[3]), int(R.shape[1])


def grid_residual(p: Params, loc: dict, vis, weight, R, grid=None):
    """Correction pass of residual_table's correction, FP64: adds to grid."""
    n = len(loc["keep"])
    Sr, OSr = _res_dims(p, R)
    if grid is None:
        grid = np.zeros((p.N, p.N), np.complex128)
    wt, wptr = _weight_arg(weight, n)
    _clib().oracle_grid_residual(n, p.N, p.S, p.OS, Sr, OSr, *_loc_args(loc), _c128(vis),
                                 wptr, _c128(R).reshape(-1),
                                 grid.view(np.float64).reshape(-1))
    return grid


def degrid_residual(p: Params, loc: dict, grid, weight, R, out=None):
    """Adjoint of grid_residual, FP64: adds to out (zeros if None)."""
    n = len(loc["keep"])
    Sr, OSr = _res_dims(p, R)
    if out is None:
        out = np.zeros(n, np.complex128)
    wt, wptr = _weight_arg(weight, n)
    _clib().oracle_degrid_residual(n, p.N, p.S, p.OS, Sr, OSr, *_loc_args(loc),
                                   _c128(grid).reshape(-1), wptr, _c128(R).reshape(-1),
                                   out.view(np.float64))
    return out


def grid(p: Params, u, v, w, vis, weight=None, T=None):
    """Locate + separable gridding of raw (u, v, w) visibilities."""
    if T is None:
        T = taps(p)
    loc = locate(p, u, v, w)
    return grid_separable(p, loc, vis, weight, T), loc


def degrid(p: Params, u, v, w, model_grid, weight=None, T=None):
    if T is None:
        T = taps(p)
    loc = locate(p, u, v, w)
    return degrid_separable(p, loc, model_grid, weight, T), loc


# --------------------------------------------------------------------------
# direct sums (definitions, tiny inputs only)
# --------------------------------------------------------------------------


def _screen_phase(w, L, M, screen, gamma):
    if screen == "exact":
        return w * n_minus_1(L, M)
    if screen == "separable":
        return w * (-0.5 * L * L - gamma * L ** 4 - 0.5 * M * M - gamma * M ** 4)
    if screen == "none":
        return 0.0 * L
    raise ValueError(screen)


def dirty_direct(N, fov, u, v, w, vis, weight=None, screen="exact",
                 gamma=5.0 / 24.0):
    """Dirty image by the direct sum of Eq. dirty:
        I_D(l, m) = n * sum_i W_i V_i exp(2 pi i (u_i l + v_i m + w_i (n-1))),
    on the N x N pixel grid l_a = nu_a fov, indexed [b][a] (m rows, l columns).
    screen='separable' replaces exp(2 pi i w (n-1)) by g~_w (Eq. gt)."""
    l = pixel_l(N, fov)
    L, M = np.meshgrid(l, l)
    n = np.sqrt(1.0 - L * L - M * M)
    wt = np.ones(len(u)) if weight is None else np.asarray(weight, np.float64)
    img = np.zeros((N, N), np.complex128)
    for i in range(len(u)):
        ph = u[i] * L + v[i] * M + _screen_phase(w[i], L, M, screen, gamma)
        img += wt[i] * complex(vis[i]) * np.exp(2j * np.pi * ph)
    return n * img


def predict_direct(N, fov, image, u, v, w, screen="exact", gamma=5.0 / 24.0):
    """Predicted visibilities by the direct sum of the prediction integral
    (Sec. 2) over the pixel grid, pixel area omitted:
        V_i = sum_{a,b} I(l_a, m_b)/n exp(-2 pi i (u_i l + v_i m + w_i (n-1)))."""
    l = pixel_l(N, fov)
    L, M = np.meshgrid(l, l)
    n = np.sqrt(1.0 - L * L - M * M)
    In = np.asarray(image, np.complex128) / n
    out = np.zeros(len(u), np.complex128)
    for i in range(len(u)):
        ph = u[i] * L + v[i] * M + _screen_phase(w[i], L, M, screen, gamma)
        out[i] = np.sum(In * np.exp(-2j * np.pi * ph))
    return out


# --------------------------------------------------------------------------
# image step with grid correction (Sec. 2)
# --------------------------------------------------------------------------


def _shift_dft_matrix(N, sign):
    a = np.arange(N, dtype=np.int64) - N // 2
    m = np.mod(np.outer(a, a), N)  # exact integer phase numerator
    return np.exp(sign * 2j * np.pi * m / N)


def _correction(p: Params, l0: float = 0.0, m0: float = 0.0):
    """n at the pixels (offset by a facet centre (l0, m0), Sec. 4.1) and the
    taper product c1(nu_a) c1(nu_b)."""
    nu = pixel_nu(p.N)
    l = nu * p.fov
    L, M = np.meshgrid(l + l0, l + m0)
    n = np.sqrt(1.0 - L * L - M * M)
    c = kb_taper(nu, p.S, p.kb_beta)
    return n, c[None, :] * c[:, None]


def grid_to_image_direct(p: Params, grid):
    """GRID -> IMAGE by the definition (direct DFT):
    I[b][a] = n / (c1(nu_a) c1(nu_b)) *
              sum_{cu,cv} grid[cv][cu] exp(2 pi i ((cu-N/2) nu_a + (cv-N/2) nu_b))."""
    E = _shift_dft_matrix(p.N, +1)
    n, cc = _correction(p)
    return n / cc * (E @ np.asarray(grid, np.complex128) @ E.T)


def grid_to_image(p: Params, grid, l0: float = 0.0, m0: float = 0.0):
    """GRID -> IMAGE with numpy.fft as the DFT primitive (same sum); for a
    facet centred at (l0, m0) the factor n is taken at l0 + l, m0 + m."""
    N = p.N
    n, cc = _correction(p, l0, m0)
    s = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(np.asarray(grid, np.complex128))))
    return n / cc * (N * N) * s


def image_to_grid_direct(p: Params, image):
    """IMAGE -> GRID (the prediction direction, Sec. 2):
    grid[cv][cu] = sum_{a,b} exp(-2 pi i ((cu-N/2) nu_a + (cv-N/2) nu_b))
                   I[b][a] / (n c1(nu_a) c1(nu_b)).
    Degridding this grid predicts V_i of the prediction integral."""
    E = _shift_dft_matrix(p.N, -1)
    n, cc = _correction(p)
    return E @ (np.asarray(image, np.complex128) / (n * cc)) @ E.T


def image_to_grid(p: Params, image):
    n, cc = _correction(p)
    x = np.asarray(image, np.complex128) / (n * cc)
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(x)))


# --------------------------------------------------------------------------
# image-plane faceting (Sec. 4.1, Eq. gt-facet)
# --------------------------------------------------------------------------


def facet_coeffs(l0: float, m0: float):
    """Quadratic coefficients of the facet screens of Eq. gt-facet:
    a_l = -(1/n0 + l0^2/n0^3)/2, a_m = -(1/n0 + m0^2/n0^3)/2, n0 = h(l0, m0).
    g^l_w(l) = exp(2 pi i w a_l l^2), g^m_w(m) = exp(2 pi i w a_m m^2)."""
    n0 = math.sqrt(1.0 - l0 * l0 - m0 * m0)
    return -0.5 * (1.0 / n0 + l0 * l0 / n0 ** 3), -0.5 * (1.0 / n0 + m0 * m0 / n0 ** 3)


def taps_facet(p: Params, l0: float, m0: float):
    """(Tu, Tv): the 1-D tables of a facet centred at (l0, m0), built as taps()
    with the screens g^l_w (u table) and g^m_w (v table) of Eq. gt-facet over
    the facet's pixels (l, m relative to the facet centre)."""
    N, S, OS = p.N, p.S, p.OS
    wp = plane_w(p.P, p.w_max)
    nu = pixel_nu(N)
    l = nu * p.fov
    c = kb_taper(nu, S, p.kb_beta)
    E = _dft_rows(S, OS, N)
    out = []
    for a in facet_coeffs(l0, m0):
        h = c[None, :] * np.exp(2j * np.pi * wp[:, None] * a * (l * l)[None, :])
        out.append(((h @ E.T) / N).reshape(len(wp), OS, S))
    return out[0], out[1]


def facet_shift(u, v, w, vis, l0: float, m0: float):
    """Visibilities of a facet (Sec. 4.1): the linear term of the Taylor
    expansion of h about (l0, m0) is absorbed by u' = u - w l0 / n0,
    v' = v - w m0 / n0, and the phase centre moves to the facet centre,
    V' = V exp(2 pi i (u l0 + v m0 + w (n0 - 1)))."""
    n0 = math.sqrt(1.0 - l0 * l0 - m0 * m0)
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    w = np.asarray(w, np.float64)
    ph = u * l0 + v * m0 + w * (n0 - 1.0)
    return u - w * l0 / n0, v - w * m0 / n0, np.asarray(vis) * np.exp(2j * np.pi * ph)


def facet_image(p: Params, l0: float, m0: float, u, v, w, vis, weight, wrap=False):
    """Dirty image of one facet: shifted visibilities gridded with the facet
    tables (separable, Sec. 5), image step with n at l0 + l, m0 + m."""
    up, vp, visp = facet_shift(u, v, w, vis, l0, m0)
    loc = locate(p, up, vp, w, wrap=wrap)
    Tu, Tv = taps_facet(p, l0, m0)
    g = grid_separable(p, loc, visp, weight, Tu, wrap=wrap, Tv=Tv)
    return grid_to_image(p, g, l0, m0)


def dirty_direct_facet(p: Params, l0: float, m0: float, u, v, w, vis, weight=None):
    """Eq. dirty over a facet's pixels (l0 + l, m0 + m) with the w term
    exp(2 pi i w (n - 1)) replaced by its facet approximation
    exp(2 pi i w (n0 - 1)) exp(-2 pi i w (l0 l + m0 m) / n0) g^l_w(l) g^m_w(m)."""
    l = pixel_l(p.N, p.fov)
    L, M = np.meshgrid(l, l)
    n = np.sqrt(1.0 - (L + l0) ** 2 - (M + m0) ** 2)
    al, am = facet_coeffs(l0, m0)
    up, vp, visp = facet_shift(u, v, w, vis, l0, m0)
    wt = np.ones(len(up)) if weight is None else np.asarray(weight, np.float64)
    img = np.zeros((p.N, p.N), np.complex128)
    for i in range(len(up)):
        ph = up[i] * L + vp[i] * M + w[i] * (al * L * L + am * M * M)
        img += wt[i] * complex(visp[i]) * np.exp(2j * np.pi * ph)
    return n * img


# --------------------------------------------------------------------------
# hybrid W stacking (Sec. 4.3)
# --------------------------------------------------------------------------


def wstack_assign(w, centres):
    """Slice of each visibility and its residual w (Sec. 4.3: visibilities
    are partitioned by w; the slice's mean w term is corrected in image space
    and the residual by W projection).

    Readings (the paper fixes no rule): the slice is the nearest centre,
    |w - w_c| compared in IEEE double, ties to the lower centre; the residual
    is w - w_c in IEEE double.  Centres must be strictly increasing.
    Non-finite w gets slice 0 and a non-finite residual (dropped later)."""
    c = np.asarray(centres, np.float64)
    if c.ndim != 1 or len(c) == 0 or np.any(np.diff(c) <= 0):
        raise ValueError("centres must be strictly increasing")
    w = np.asarray(w, np.float64)
    with np.errstate(invalid="ignore"):
        d = np.abs(w[:, None] - c[None, :])
    d = np.where(np.isnan(d), np.inf, d)
    layer = np.argmin(d, axis=1)  # first minimum: ties to the lower centre
    return layer, w - c[layer]


def wstack_phase(p: Params, wc: float):
    """Image-space phase of a slice centre, exp(2 pi i w_c (n - 1)), on the
    pixel grid [b][a] (the w term of Eq. dirty for w = w_c)."""
    l = pixel_l(p.N, p.fov)
    L, M = np.meshgrid(l, l)
    return np.exp(2j * np.pi * wc * n_minus_1(L, M))


def wstack_layer_grids(p: Params, u, v, w, vis, weight, centres, T=None, wrap=False,
                       kernel: str = "separable"):
    """Per-slice grids of the residual w: separable gridding (Sec. 5) of the
    visibilities of each slice with their residual w, or with the exact 2-D
    kernel (kernel='exact', for the pins).  Returns (grids [slice][N][N],
    slice of each visibility, residual w)."""
    layer, wr = wstack_assign(w, centres)
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    vis = np.asarray(vis)
    wt = None if weight is None else np.asarray(weight, np.float64)
    if kernel == "separable":
        K = taps(p) if T is None else T
    else:
        K = exact_table(p) if T is None else T
    grids = np.zeros((len(centres), p.N, p.N), np.complex128)
    for c in range(len(centres)):
        sel = layer == c
        if not np.any(sel):
            continue
        loc = locate(p, u[sel], v[sel], wr[sel], wrap=wrap)
        ws = None if wt is None else wt[sel]
        if kernel == "separable":
            grids[c] = grid_separable(p, loc, vis[sel], ws, K, wrap=wrap)
        else:
            grids[c] = grid_exact2d(p, loc, vis[sel], ws, K, wrap=wrap)
    return grids, layer, wr


def wstack_image(p: Params, u, v, w, vis, weight, centres, T=None, wrap=False,
                 kernel: str = "separable"):
    """Dirty image by hybrid W stacking (Sec. 4.3): for every slice, the image
    step (Sec. 2) of its residual-w grid times the slice centre's phase
    exp(2 pi i w_c (n - 1)), summed over the slices."""
    grids, _, _ = wstack_layer_grids(p, u, v, w, vis, weight, centres, T, wrap, kernel)
    img = np.zeros((p.N, p.N), np.complex128)
    for c, wc in enumerate(centres):
        img += grid_to_image(p, grids[c]) * wstack_phase(p, wc)
    return img


def wstack_model_grids(p: Params, image, centres):
    """Prediction direction of hybrid W stacking: for every slice the model
    image times exp(-2 pi i w_c (n - 1)), then IMAGE -> GRID (Sec. 2).
    Degridding slice c's grid with the residual w of its visibilities
    predicts them (the prediction integral with w = w_c + residual)."""
    img = np.asarray(image, np.complex128)
    return np.stack([image_to_grid(p, img * np.conj(wstack_phase(p, wc))) for wc in centres])


# --------------------------------------------------------------------------
# major cycles: weighted least-squares imaging by conjugate gradients
# --------------------------------------------------------------------------


def predict_op(p: Params, loc: dict, T, image):
    """M x: IMAGE -> GRID (Sec. 2) then separable degridding with unit
    weights: the visibilities predicted from a model image."""
    return degrid_separable(p, loc, image_to_grid(p, image), None, T)


def predict_adjoint(p: Params, loc: dict, T, vis):
    """M^H r: separable gridding with unit weights, then the adjoint of
    IMAGE -> GRID, which is GRID -> IMAGE divided by n^2."""
    g = grid_separable(p, loc, vis, None, T)
    l = pixel_l(p.N, p.fov)
    L, M = np.meshgrid(l, l)
    return grid_to_image(p, g) / (1.0 - L * L - M * M)


def cg_major_cycles(p: Params, loc: dict, T, vis, weight, n_cycles: int, x0=None):
    """Weighted least-squares imaging, min over real images x of
    sum_i W_i |(M x)_i - V_i|^2, by conjugate gradients on the normal
    equations.  Each cycle predicts the visibilities of a search direction
    (degridding) and grids them back (gridding): the alternation of major
    cycles (Sec. 6), with the model update of least squares in place of a
    CLEAN minor cycle.

    Reading (the paper gives no solver): CG runs on y with x = D y,
    D = n c1(nu_a) c1(nu_b) the grid correction, i.e. on the operator M D,
    which is prediction without the division by n c1 c1.  M itself divides
    by n c1 c1, up to 1e8 at the image edge for support 16, and unpreconditioned
    CG loses conjugacy there.

    Returns (x, losses, residuals r_k, directions d_k) with losses[k] the
    weighted chi^2 after k cycles and r_k, d_k the CG vectors in y."""
    vis = np.asarray(vis, np.complex128)
    wt = np.ones(len(vis)) if weight is None else np.asarray(weight, np.float64)
    n, cc = _correction(p)
    D = n * cc
    y = np.zeros((p.N, p.N)) if x0 is None else np.array(x0, np.float64) / D

    def op(y_):  # M D y
        return predict_op(p, loc, T, D * y_)

    def op_h(r_):  # Re(D M^H r)
        return D * predict_adjoint(p, loc, T, r_).real

    def loss(y_):
        r_ = op(y_) - vis
        return float(np.sum(wt * (r_.real ** 2 + r_.imag ** 2)))

    r = op_h(wt * (vis - op(y)))
    d = r.copy()
    rr = float(np.sum(r * r))
    losses, rs, ds = [loss(y)], [r.copy()], [d.copy()]
    for _ in range(n_cycles):
        q = op_h(wt * op(d))
        alpha = rr / float(np.sum(d * q))
        y = y + alpha * d
        r = r - alpha * q
        rr_new = float(np.sum(r * r))
        d = r + (rr_new / rr) * d
        rr = rr_new
        losses.append(loss(y))
        rs.append(r.copy())
        ds.append(d.copy())
    return D * y, losses, rs, ds


# --------------------------------------------------------------------------
# analysis formulas (Secs. 2-4, Appendix A)
# --------------------------------------------------------------------------


def eps_leading(l, m, gamma):
    """Leading-order phase error factor of Sec. 3:
    eps = (1/8 - gamma)(l^4 + m^4) + l^2 m^2 / 4."""
    return (0.125 - gamma) * (l ** 4 + m ** 4) + 0.25 * l * l * m * m


def eps_exact(l, m, gamma):
    """Exact phase error factor of g~ against g (Sec. 3, before expansion):
    eps = -(l^2/2 + gamma l^4 + m^2/2 + gamma m^4) - (n - 1)."""
    return -(0.5 * l * l + gamma * l ** 4 + 0.5 * m * m + gamma * m ** 4) - n_minus_1(l, m)


def errscale(Q, lam, D, B, elevation_rad):
    """Eq. errscale: |dl| / theta_res ~ (1/18) Q^4 lambda^3 D^-4 B cot(a)."""
    return Q ** 4 * lam ** 3 * B / (18.0 * D ** 4 * math.tan(elevation_rad))


def w_support(w, fov, eta):
    """Support (uv cells) of the W kernel truncated at eta of its peak (Sec. 2):
    2 fov sqrt((w fov / 2)^2 + w^(3/2) fov / (2 pi eta))."""
    return 2 * fov * np.sqrt((w * fov / 2) ** 2 + w ** 1.5 * fov / (2 * np.pi * eta))


def n_wplanes_needed(w_max, fov, dA):
    """Number of w planes of Sec. 2: pi w_max fov^2 / sqrt(2 dA)."""
    return np.pi * w_max * fov ** 2 / math.sqrt(2 * dA)


def amplitude_loss(eps, w_max):
    """Eq. amplitude-loss: expected loss 2/3 pi^2 eps^2 w_max^2 for residual
    dw uniform in [-w_max, w_max]."""
    return 2.0 / 3.0 * np.pi ** 2 * eps ** 2 * w_max ** 2


def delta_l_roots(l, d, eps):
    """Appendix A: exact dl = y d from the quadratic
    (1 + |d|^2) y^2 + 2 (l.d - k) y + (2n + eps) eps = 0, k = n + eps;
    returns the root of smaller magnitude."""
    l = np.asarray(l, np.float64)
    d = np.asarray(d, np.float64)
    n = math.sqrt(1.0 - float(l @ l))
    k = n + eps
    a = 1.0 + float(d @ d)
    b = 2.0 * (float(l @ d) - k)
    c = (2.0 * n + eps) * eps
    disc = math.sqrt(b * b - 4 * a * c)
    q = -0.5 * (b + math.copysign(disc, b))
    roots = [q / a, c / q]
    return min(roots, key=abs)


def delta_l_y1(l, d, eps):
    """Appendix A first-order approximation y1 = (1 + l.d / n) eps."""
    l = np.asarray(l, np.float64)
    d = np.asarray(d, np.float64)
    n = math.sqrt(1.0 - float(l @ l))
    return (1.0 + float(l @ d) / n) * eps


__all__ = [name for name, val in list(globals().items())
           if not name.startswith("_") and not isinstance(val, type(math))]
