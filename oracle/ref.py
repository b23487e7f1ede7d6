"""CPU FP64 oracle for OptA template search -- TEST INFRASTRUCTURE ONLY.

Only tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may call this module.  It shares no code with the CUDA library.

What the search computes has a plain definition, so the graded oracle is
that definition written out (Section 1, Eq. rho1):

    rho(y, x) = sum_{u,v} (t(u,v) - mu_t)(I(y+u, x+v) - mu_o) / (sigma_t sigma_o)

at every location, in FP64, and the best match is the argmax of rho with
ties broken towards the lowest row-major index.  ``rho := 0`` for a flat
window (sigma == 0).

The preparation steps (blur, blur-correlation, auto-correlation, EGS and
the OptA level loop) only decide how much work the search skips, never its
answer; they are written here in the paper's order for diagnostic parity:

* ``blur``            -- Eq. defblur / Eq. Gauss, per-block sigma.
* ``blur_corr_map``   -- R_oo of Algorithm 3.
* ``rho_co_map``      -- Algorithm 1 (pivot = blurred centre block).
* ``egs``             -- Algorithm 2 with Eq. co's retained count.
* ``opta``            -- Algorithm 3 under the readings stated in its docstring.

The paper's own procedure (Section 4.3), which searches the blurred image
and re-matches locally, is written out too (``opta_literal``,
``literal_search``).  Its answer is not the exact maximum in general; it is
pinned through the cases where it must be (no blur, or a neighbourhood that
covers every location), and how far it lands from the maximum otherwise is
measured, not pinned (the paper's images are not available).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    """Load (building if needed) the oracle's C routines."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i64 = ctypes.c_int64
        ci = ctypes.c_int
        L.oracle_window_rho.restype = ctypes.c_double
        L.oracle_window_rho.argtypes = [dp, i64, dp, i64, ci, ci, ci, ci, ci, ci]
        L.oracle_zncc_map.restype = None
        L.oracle_zncc_map.argtypes = [dp, i64, ci, ci, dp, ci, ci, dp, ci]
        L.oracle_rho_at.restype = None
        L.oracle_rho_at.argtypes = [dp, i64, dp, ci, ci, ip, ip, ci, dp, ci]
        L.oracle_blur_corr_map.restype = None
        L.oracle_blur_corr_map.argtypes = [dp, dp, i64, ci, ci, ci, ci, dp, ci]
        L.oracle_rho_co_map.restype = None
        L.oracle_rho_co_map.argtypes = [dp, dp, i64, ci, ci, ci, ci, ci, dp, ci]
        L.oracle_blur.restype = None
        L.oracle_blur.argtypes = [dp, i64, ci, ci, dp, ci, dp, ci]
        L.oracle_max_threads.restype = ci
        L.oracle_max_threads.argtypes = []
        _LIB = L
    return _LIB


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


# ---------------------------------------------------------------------------
# Eq. rho1: correlation coefficient
# ---------------------------------------------------------------------------
def rho_pair(a: np.ndarray, b: np.ndarray) -> float:
    """rho between two equal-shape blocks, two-pass FP64 (Eq. rho1)."""
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    da = a - a.mean(); db = b - b.mean()
    va = float((da * da).sum()); vb = float((db * db).sum())
    if va == 0.0 or vb == 0.0:
        return 0.0
    return float((da * db).sum()) / (math.sqrt(va) * math.sqrt(vb))


def rho_direct(img: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Eq. rho1 at every location with pure-Python loops (tiny inputs only)."""
    img = np.asarray(img, dtype=np.float64); t = np.asarray(t, dtype=np.float64)
    m, n = t.shape; p, q = img.shape
    out = np.zeros((p - m + 1, q - n + 1))
    for y in range(p - m + 1):
        for x in range(q - n + 1):
            out[y, x] = rho_pair(t, img[y:y + m, x:x + n])
    return out


def zncc_map(img: np.ndarray, t: np.ndarray, threads: int = 0) -> np.ndarray:
    """Eq. rho1 at every location (C, FP64, OpenMP over rows)."""
    I, Ip = _d(img); T, Tp = _d(t)
    p, q = I.shape; m, n = T.shape
    if m > p or n > q:
        raise ValueError("template larger than image")
    out = np.empty((p - m + 1, q - n + 1), dtype=np.float64)
    lib().oracle_zncc_map(Ip, q, p, q, Tp, m, n,
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), threads)
    return out


def zncc_map_fft(img: np.ndarray, t: np.ndarray, workers: int = -1) -> np.ndarray:
    """Eq. rho1 at every location, for images too large for the direct loop.

    The numerator sum_{u,v} t'(u,v) I(y+u, x+v), with t' = t - mu_t (its sum
    is zero, so the window mean of I drops out), is one cross-correlation,
    taken here with a library FFT in FP64 over the whole image (no location
    reaches past the image, so the transform's wrap-around never enters).
    The window sums S and Q of I come from integral images; for integer
    images they are exact int64, so sigma_o^2 = (mn Q - S^2) / mn is exact up
    to its final rounding and a flat window is recognised exactly (rho := 0).
    The FFT's rounding error is of order 1e-16 log2(pq) ||t'|| ||I - 128||,
    far below the 1e-6 that the tests resolve."""
    return next(zncc_maps_fft(img, [t], workers))


def zncc_maps_fft(img: np.ndarray, templates, workers: int = -1):
    """``zncc_map_fft`` for several templates of one image, yielding one map
    per template in order (the image's transform and integral images are
    taken once)."""
    from scipy import fft as sfft
    I = np.asarray(img, dtype=np.float64)
    p, q = I.shape
    F_I = sfft.rfft2(I - 128.0, workers=workers)
    exact = bool(np.all(I == np.rint(I)) and np.abs(I).max() < 2 ** 20)
    if exact:
        Ii = I.astype(np.int64)
        iis = np.zeros((p + 1, q + 1), dtype=np.int64)
        iiq = np.zeros((p + 1, q + 1), dtype=np.int64)
        iis[1:, 1:] = Ii.cumsum(0).cumsum(1)
        iiq[1:, 1:] = (Ii * Ii).cumsum(0).cumsum(1)
        del Ii
    else:
        iis = np.zeros((p + 1, q + 1)); iiq = np.zeros((p + 1, q + 1))
        iis[1:, 1:] = I.cumsum(0).cumsum(1)
        iiq[1:, 1:] = (I * I).cumsum(0).cumsum(1)
    var_of = {}
    for t in templates:
        T = np.asarray(t, dtype=np.float64)
        m, n = T.shape
        if m > p or n > q:
            raise ValueError("template larger than image")
        Ly, Lx = p - m + 1, q - n + 1
        mn = m * n
        if (m, n) not in var_of:
            S = iis[m:, n:] - iis[:Ly, n:] - iis[m:, :Lx] + iis[:Ly, :Lx]
            Q = iiq[m:, n:] - iiq[:Ly, n:] - iiq[m:, :Lx] + iiq[:Ly, :Lx]
            if exact:
                var = (mn * Q - S * S).astype(np.float64) / mn
            else:
                var = np.maximum(Q - S * S / mn, 0.0)
            var_of = {(m, n): var}          # one size at a time is kept
        var = var_of[(m, n)]
        tz = T - T.mean()
        st = math.sqrt(float((tz * tz).sum()))
        out = np.zeros((Ly, Lx))
        if st > 0.0:
            pad = np.zeros((p, q))
            pad[:m, :n] = tz
            F = np.conj(sfft.rfft2(pad, workers=workers))
            del pad
            F *= F_I
            num = sfft.irfft2(F, s=(p, q), workers=workers)[:Ly, :Lx]
            del F
            ok = var > 0
            out[ok] = num[ok] / (st * np.sqrt(var[ok]))
        yield out


def rho_at(img: np.ndarray, t: np.ndarray, ys, xs, threads: int = 0) -> np.ndarray:
    """Eq. rho1 at the listed locations (C, FP64)."""
    I, Ip = _d(img); T, Tp = _d(t)
    p, q = I.shape; m, n = T.shape
    ys = np.ascontiguousarray(ys, dtype=np.int32); xs = np.ascontiguousarray(xs, dtype=np.int32)
    if ys.size and (ys.min() < 0 or xs.min() < 0 or ys.max() > p - m or xs.max() > q - n):
        raise ValueError("location out of range")
    out = np.empty(ys.size, dtype=np.float64)
    ip = ctypes.POINTER(ctypes.c_int)
    lib().oracle_rho_at(Ip, q, Tp, m, n, ys.ctypes.data_as(ip), xs.ctypes.data_as(ip),
                        int(ys.size), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), threads)
    return out


def argmax_first(rho: np.ndarray):
    """(y, x, value) of the maximum; ties -> lowest row-major index."""
    k = int(np.argmax(rho))          # numpy returns the first occurrence
    y, x = divmod(k, rho.shape[1])
    return y, x, float(rho[y, x])


def best_match(img, t, threads: int = 0):
    """The graded result: argmax of Eq. rho1 over all locations."""
    return argmax_first(zncc_map(img, t, threads))


# ---------------------------------------------------------------------------
# Section 2: transitive bounds
# ---------------------------------------------------------------------------
def transitive_upper(r_tc, r_co):
    """Eq. tranEqq: rho_to <= rho_tc rho_co + sqrt((1-rho_tc^2)(1-rho_co^2))."""
    r_tc = np.asarray(r_tc, dtype=np.float64); r_co = np.asarray(r_co, dtype=np.float64)
    return r_tc * r_co + np.sqrt(np.clip((1 - r_tc ** 2) * (1 - r_co ** 2), 0, None))


def transitive_lower(r_tc, r_co):
    """Lower transitive bound (Section 2): rho_tc rho_co - sqrt(...)."""
    r_tc = np.asarray(r_tc, dtype=np.float64); r_co = np.asarray(r_co, dtype=np.float64)
    return r_tc * r_co - np.sqrt(np.clip((1 - r_tc ** 2) * (1 - r_co ** 2), 0, None))


def transitive_gap(r_tc, r_co):
    """Eq. eps: epsilon = 2 sqrt(1-rho_tc^2) sqrt(1-rho_co^2)."""
    r_tc = np.asarray(r_tc, dtype=np.float64); r_co = np.asarray(r_co, dtype=np.float64)
    return 2.0 * np.sqrt(1 - r_tc ** 2) * np.sqrt(1 - r_co ** 2)


def lam(rho_th: float, rho_max: float) -> float:
    """Eq. misDec: the blur-correlation level below which a region stays unblurred."""
    return rho_th * rho_max + math.sqrt(
        max(0.0, 1.0 + rho_th ** 2 * rho_max ** 2 - (rho_th ** 2 + rho_max ** 2)))


def egs_rho_cut(rho_th: float) -> float:
    """Proposition 3.2 / Eq. co: a location counts as retained if rho_co < sqrt(1-rho_th^2)."""
    return math.sqrt(1.0 - rho_th * rho_th)


# ---------------------------------------------------------------------------
# Group layout (Fig. 1, Section 2; reading of Algorithm 1's indexing)
# ---------------------------------------------------------------------------
def group_centre(c: int, length: int, h: int) -> int:
    start = (c // h) * h
    size = min(h, length - start)
    return start + (size - 1) // 2


def group_centres_axis(length: int, h: int) -> np.ndarray:
    """Centre coordinates of the groups along one axis of `length` locations."""
    starts = np.arange(0, length, h)
    sizes = np.minimum(h, length - starts)
    return starts + (sizes - 1) // 2


def n_groups(Ly: int, Lx: int, h: int) -> int:
    return ((Ly + h - 1) // h) * ((Lx + h - 1) // h)


# ---------------------------------------------------------------------------
# Section 4: blur, Section 5 / Algorithm 3: blur-correlation
# ---------------------------------------------------------------------------
def blur_support(sigma: float) -> int:
    """Reading of Section 4's filter size: d = ceil(3 sigma)."""
    return int(math.ceil(3.0 * sigma)) if sigma > 0 else 0


def blur(img: np.ndarray, sigma_map: np.ndarray, block: int, threads: int = 0) -> np.ndarray:
    """Eq. defblur with Eq. Gauss weights, sigma per output pixel's block (C, FP64)."""
    I, Ip = _d(img); S, Sp = _d(sigma_map)
    p, q = I.shape
    if S.shape != ((p + block - 1) // block, (q + block - 1) // block):
        raise ValueError("sigma_map shape does not match the image blocks")
    out = np.empty((p, q), dtype=np.float64)
    lib().oracle_blur(Ip, q, p, q, Sp, block,
                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), threads)
    return out


def quantise_pivot(blurred: np.ndarray) -> np.ndarray:
    """Pivot image: round half to even to the nearest integer (uint8 range)."""
    return np.clip(np.rint(blurred), 0, 255).astype(np.uint8)


def blur_corr_map(P: np.ndarray, I: np.ndarray, m: int, n: int, threads: int = 0) -> np.ndarray:
    """R_oo(x) = rho(P window at x, I window at x) (Algorithm 3)."""
    A, Ap = _d(P); B, Bp = _d(I)
    p, q = B.shape
    out = np.empty((p - m + 1, q - n + 1))
    lib().oracle_blur_corr_map(Ap, Bp, q, p, q, m, n,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), threads)
    return out


def rho_co_map(P: np.ndarray, I: np.ndarray, m: int, n: int, h: int, threads: int = 0) -> np.ndarray:
    """Algorithm 1 in pivot form: rho(P window at the group centre, I window at x)."""
    A, Ap = _d(P); B, Bp = _d(I)
    p, q = B.shape
    out = np.empty((p - m + 1, q - n + 1))
    lib().oracle_rho_co_map(Ap, Bp, q, p, q, m, n, h,
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), threads)
    return out


def flat_windows(img: np.ndarray, m: int, n: int) -> np.ndarray:
    """Boolean map: window at x is flat (all pixels equal)."""
    from numpy.lib.stride_tricks import sliding_window_view
    w = sliding_window_view(np.asarray(img, dtype=np.float64), (m, n))
    return w.max(axis=(2, 3)) == w.min(axis=(2, 3))


# ---------------------------------------------------------------------------
# Section 3: EGS (Algorithm 2)
# ---------------------------------------------------------------------------
EGS_RUN = 8   # group rows per run of EGS's systematic sample


def egs_sample_rows(Ly: int, h: int, sample: int = 1) -> np.ndarray:
    """Boolean mask of the location rows EGS counts for group side h: the
    rows of the group rows g with (g // EGS_RUN) % sample == 0 (every row
    when sample <= 1).  Reading: Algorithm 2's n_r only steers the choice of
    h and blur level, so it may be estimated from a systematic sample of the
    location grid; sample = 1 is the count as printed."""
    g = np.arange(Ly) // h
    if sample <= 1:
        return np.ones(Ly, dtype=bool)
    return (g // EGS_RUN) % sample == 0


def egs_cost(rco: np.ndarray, h: int, rho_th: float, sample: int = 1) -> int:
    """Total estimated cost in units of one rho evaluation (Section 3.3, Eq. objfunc):
    number of groups (centre evaluations) + retained count n_r (Eq. co, strict `<`
    as in Algorithm 2).  With sample > 1, n_r is counted over the sampled rows and
    scaled by Ly / (rows sampled), rounded to the nearest integer (halves up)."""
    Ly, Lx = rco.shape
    rows = egs_sample_rows(Ly, h, sample)
    cnt = int(np.count_nonzero(rco[rows] < egs_rho_cut(rho_th)))
    ns = int(rows.sum())
    n_r = (cnt * Ly + ns // 2) // ns
    return n_groups(Ly, Lx, h) + n_r


def egs(P, I, m, n, h_start, rho_th, xi, h_max=9, threads=0, log=None, sample=1):
    """Algorithm 2: grow the square group size by 2 while the cost falls by more
    than the fraction xi of the previous cost; returns (h_e, cost_e)."""
    h = h_start
    c_prev = egs_cost(rho_co_map(P, I, m, n, h, threads), h, rho_th, sample)
    if log is not None:
        log.append((h, c_prev))
    while h + 2 <= h_max:
        c_new = egs_cost(rho_co_map(P, I, m, n, h + 2, threads), h + 2, rho_th, sample)
        if log is not None:
            log.append((h + 2, c_new))
        if c_prev - c_new > xi * c_prev:
            h, c_prev = h + 2, c_new
        else:
            break
    return h, c_prev


# ---------------------------------------------------------------------------
# Section 5: OptA (Algorithm 3), per-block Gaussian levels
# ---------------------------------------------------------------------------
DEFAULT_LEVELS = (0.5, 1.0, 2.0, 3.0)


def opta(I, m, n, rho_th=0.8, rho_max=0.95, xi=0.005, block=64,
         levels=DEFAULT_LEVELS, h_max=9, threads=0, literal=False, sample=1):
    """Algorithm 3 under the reading: level k raises every still-active block to
    sigma_k; a block whose windows (by top-left, non-flat I windows only) reach
    a blur-correlation below lambda (Eq. misDec) reverts to its previous sigma
    and is frozen; the level is kept if EGS's cost falls by more than xi.
    With literal=True, EGS measures rho(P, P) (see ``opta_literal``); sample
    is EGS's count sample (``egs_sample_rows``).

    Returns dict(sigma_map, pivot (uint8), h, cost, trace).  Each trace entry
    after level 0 also holds the blocks that failed the lambda test at that
    level (``fail``) and the frozen blocks after it (``frozen_map``)."""
    I = np.asarray(I, dtype=np.float64)
    p, q = I.shape
    bp, bq = (p + block - 1) // block, (q + block - 1) // block
    lamb = lam(rho_th, rho_max)
    sig = np.zeros((bp, bq))
    frozen = np.zeros((bp, bq), dtype=bool)
    P = quantise_pivot(I)
    h, cost = egs(P, P if literal else I, m, n, 1, rho_th, xi, h_max, threads, sample=sample)
    trace = [dict(level=0, sigma=0.0, h=h, cost=cost, frozen=0)]
    flat = flat_windows(I, m, n)
    Ly, Lx = p - m + 1, q - n + 1
    by = (np.arange(Ly) // block)[:, None]
    bx = (np.arange(Lx) // block)[None, :]
    for k, s in enumerate(levels, start=1):
        if frozen.all():
            break
        cand = np.where(frozen, sig, s)
        Pk = quantise_pivot(blur(I, cand, block, threads))
        R = blur_corr_map(Pk, I, m, n, threads)
        bad = (R < lamb) & ~flat
        fail = np.zeros((bp, bq), dtype=bool)
        np.logical_or.at(fail, (np.broadcast_to(by, bad.shape)[bad], np.broadcast_to(bx, bad.shape)[bad]), True)
        fail &= ~frozen
        new_sig = np.where(fail, sig, cand)
        new_frozen = frozen | fail
        if fail.any():
            Pk = quantise_pivot(blur(I, new_sig, block, threads))
        hk, ck = egs(Pk, Pk if literal else I, m, n, h, rho_th, xi, h_max, threads, sample=sample)
        trace.append(dict(level=k, sigma=s, h=hk, cost=ck, frozen=int(new_frozen.sum()),
                          fail=fail.copy(), frozen_map=new_frozen.copy()))
        if cost - ck > xi * cost:
            sig, frozen, P, h, cost = new_sig, new_frozen, Pk, hk, ck
        else:
            break
    return dict(sigma_map=sig, pivot=P, h=h, cost=cost, trace=trace)


# ---------------------------------------------------------------------------
# Section 4.3 as printed: search the blurred image, re-match locally on I
# ---------------------------------------------------------------------------
def opta_literal(I, m, n, **kw):
    """Algorithm 3 as Section 4.3 uses it: EGS measures the blurred image's own
    auto-correlation, rho(centre window of P, member window of P), instead of
    the pivot form rho(P, I).  Same level loop and return value as ``opta``."""
    return opta(I, m, n, literal=True, **kw)


def literal_support(sigma_map) -> int:
    """Half-width d of the re-match neighbourhood: the blur support (Section
    4.3 uses the (2d+1) x (2d+1) filter size) of the largest sigma applied."""
    s = float(np.max(sigma_map)) if np.size(sigma_map) else 0.0
    return blur_support(s)


def literal_search(I, P, t, d, threads=0):
    """Section 4.3: the best match of t on the blurred image P (exact argmax
    over P, ties to the lowest row-major index), then t matched with I in the
    (2d+1) x (2d+1) neighbourhood of that location (clipped to the location
    grid), FP64, same tie rule.  Returns (y, x, rho on I, y_hat, x_hat)."""
    rP = zncc_map(P, t, threads)
    yh, xh, _ = argmax_first(rP)
    Ly, Lx = rP.shape
    y0, y1 = max(0, yh - d), min(Ly, yh + d + 1)
    x0, x1 = max(0, xh - d), min(Lx, xh + d + 1)
    ys, xs = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    vals = rho_at(I, t, ys.ravel(), xs.ravel(), threads).reshape(ys.shape)
    wy, wx, best = argmax_first(vals)
    return y0 + wy, x0 + wx, best, yh, xh

