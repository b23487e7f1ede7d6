"""Pins for the CPU FP64 oracle, checked against things other than itself:
exact rational arithmetic, closed forms, invariants, library routines and the
values the paper prints.  CPU only."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import ref
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# Eq. rho1 against exact rational arithmetic
# ---------------------------------------------------------------------------
def _rho_fraction(t, r):
    """Exact rho^2 and sign with Python Fractions (no floating point)."""
    t = [Fraction(int(v)) for v in np.asarray(t).ravel()]
    r = [Fraction(int(v)) for v in np.asarray(r).ravel()]
    k = len(t)
    mt = sum(t) / k; mr = sum(r) / k
    num = sum((a - mt) * (b - mr) for a, b in zip(t, r))
    vt = sum((a - mt) ** 2 for a in t); vr = sum((b - mr) ** 2 for b in r)
    if vt == 0 or vr == 0:
        return Fraction(0), 0
    return num * num / (vt * vr), (1 if num > 0 else (-1 if num < 0 else 0))


def test_rho_matches_exact_rationals():
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=(11, 12)).astype(np.float64)
    img[2:6, 3:7] = 17.0                       # a flat patch
    t = rng.integers(0, 256, size=(3, 4)).astype(np.float64)
    got_c = ref.zncc_map(img, t)
    got_py = ref.rho_direct(img, t)
    for y in range(img.shape[0] - 2):
        for x in range(img.shape[1] - 3):
            r2, sgn = _rho_fraction(t, img[y:y + 3, x:x + 4])
            exact = sgn * math.sqrt(float(r2))
            assert abs(got_c[y, x] - exact) < 1e-13
            assert abs(got_py[y, x] - exact) < 1e-13
    # the flat window got rho := 0
    assert got_c[2, 3] == 0.0


def test_rho_is_one_at_exact_crop_and_is_argmax():
    img = synth.white_blur_image(64, seed=3)
    y0, x0 = 23, 31
    t = img[y0:y0 + 9, x0:x0 + 7].copy()
    rho = ref.zncc_map(img, t)
    assert abs(rho[y0, x0] - 1.0) < 1e-12
    y, x, v = ref.argmax_first(rho)
    assert (y, x) == (y0, x0)


@pytest.mark.parametrize("a,b", [(1.7, -40.0), (0.3, 900.0), (-2.0, 5.0)])
def test_affine_intensity_invariance(a, b):
    img = synth.white_blur_image(48, seed=11)
    t = synth.white_blur_image(48, seed=12)[5:13, 9:19].astype(np.float64)
    base = ref.zncc_map(img, t)
    moved = ref.zncc_map(img, a * t + b)
    assert np.allclose(moved, np.sign(a) * base, atol=1e-12)


def test_symmetry_and_range():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(20, 20)); B = rng.normal(size=(20, 20))
    L = ref.lib()
    Ap = A.ctypes.data_as(ref.ctypes.POINTER(ref.ctypes.c_double))
    Bp = B.ctypes.data_as(ref.ctypes.POINTER(ref.ctypes.c_double))
    r1 = L.oracle_window_rho(Ap, 20, Bp, 20, 6, 5, 1, 2, 7, 3)
    r2 = L.oracle_window_rho(Bp, 20, Ap, 20, 6, 5, 7, 3, 1, 2)
    assert r1 == pytest.approx(r2, abs=1e-15)
    rho = ref.zncc_map(A, B[:5, :5])
    assert np.all(np.abs(rho) <= 1.0 + 1e-15)


def test_single_location_equals_numpy_corrcoef():
    rng = np.random.default_rng(9)
    A = rng.normal(size=(13, 17)); T = rng.normal(size=(13, 17))
    rho = ref.zncc_map(A, T)
    assert rho.shape == (1, 1)
    assert rho[0, 0] == pytest.approx(np.corrcoef(A.ravel(), T.ravel())[0, 1], abs=1e-14)


def test_rho_at_matches_map():
    img = synth.white_blur_image(40, seed=2)
    t = img[3:11, 4:12] * 1.1 + 3.0
    rho = ref.zncc_map(img, t)
    ys = np.array([0, 5, 32, 17]); xs = np.array([0, 30, 32, 4])
    assert np.allclose(ref.rho_at(img, t, ys, xs), rho[ys, xs], atol=0, rtol=0)


def test_null_distribution_mean_rho_squared():
    """Section 3 (Proposition 3.2's proof): for uncorrelated Gaussian data the
    mean of rho^2 is 1/(mn-1)."""
    rng = np.random.default_rng(123)
    img = rng.normal(size=(400, 400))
    t = rng.normal(size=(4, 4))
    # use non-overlapping windows so the samples are independent
    rho = ref.zncc_map(img, t)[::4, ::4].ravel()
    mn = 16
    mean = float(np.mean(rho ** 2))
    # Var(rho^2) for Beta(1/2, (mn-2)/2): a=1/2, b=(mn-2)/2
    a, b = 0.5, (mn - 2) / 2.0
    var = a * b / ((a + b) ** 2 * (a + b + 1))
    se = math.sqrt(var / rho.size)
    assert abs(mean - 1.0 / (mn - 1)) < 5 * se


def test_brute_force_argmax_tiny():
    rng = np.random.default_rng(31)
    img = rng.integers(0, 256, size=(9, 10)).astype(float)
    t = rng.integers(0, 256, size=(3, 3)).astype(float)
    rho = ref.rho_direct(img, t)
    best = max((rho[y, x], -(y * rho.shape[1] + x)) for y in range(rho.shape[0]) for x in range(rho.shape[1]))
    k = -best[1]
    assert ref.argmax_first(ref.zncc_map(img, t))[:2] == divmod(k, rho.shape[1])


def test_argmax_ties_lowest_index():
    rho = np.array([[0.1, 0.9, 0.2], [0.9, 0.3, 0.9]])
    assert ref.argmax_first(rho) == (0, 1, 0.9)


# ---------------------------------------------------------------------------
# Section 2: transitive bounds
# ---------------------------------------------------------------------------
def test_fig2_worked_example():
    for rco, r2, lo, hi, dec in _golden_rows("fig2_bounds.txt"):
        rco, r2, lo, hi, dec = float(rco), float(r2), float(lo), float(hi), int(dec)
        assert round(float(ref.transitive_upper(r2, rco)), dec) == hi
        assert round(float(ref.transitive_lower(r2, rco)), dec) == lo
        # the gap of Eq. eps is the distance between the two
        assert float(ref.transitive_gap(r2, rco)) == pytest.approx(
            float(ref.transitive_upper(r2, rco) - ref.transitive_lower(r2, rco)), abs=1e-15)


def test_bounds_are_cosine_of_angle_difference():
    """Closed form: the bounds are cos(acos a -/+ acos b)."""
    g = np.linspace(-1, 1, 41)
    A, B = np.meshgrid(g, g)
    assert np.allclose(ref.transitive_upper(A, B), np.cos(np.abs(np.arccos(A) - np.arccos(B))), atol=1e-12)
    assert np.allclose(ref.transitive_lower(A, B), np.cos(np.arccos(A) + np.arccos(B)), atol=1e-12)
    # tight when the middle block is the outer block itself
    assert np.allclose(ref.transitive_upper(g, np.ones_like(g)), g, atol=1e-12)


def test_transitive_bounds_hold_on_real_triples():
    """For every triple (t, c, o) of blocks, rho_to lies between the bounds."""
    img = synth.white_blur_image(72, seed=21)
    rng = np.random.default_rng(4)
    m = n = 8
    L = img.shape[0] - m + 1
    t = synth.white_blur_image(72, seed=22)[10:18, 30:38]
    for _ in range(300):
        cy, cx, oy, ox = rng.integers(0, L, size=4)
        c = img[cy:cy + m, cx:cx + n]; o = img[oy:oy + m, ox:ox + n]
        rtc = ref.rho_pair(t, c); rco = ref.rho_pair(c, o); rto = ref.rho_pair(t, o)
        assert rto <= ref.transitive_upper(rtc, rco) + 1e-12
        assert rto >= ref.transitive_lower(rtc, rco) - 1e-12


def test_lambda_closed_form_and_paper_parameters():
    p = {r[0]: float(r[1]) for r in _golden_rows("opta_params.txt")}
    rth, rmax = p["rho_th"], p["rho_max_reported"]
    # Eq. misDec equals cos(acos rho_max - acos rho_th)
    assert ref.lam(rth, rmax) == pytest.approx(math.cos(math.acos(rmax) - math.acos(rth)), abs=1e-14)
    assert ref.lam(rth, 1.0) == pytest.approx(rth, abs=1e-15)
    assert round(ref.lam(rth, rmax), 6) == 0.947350
    assert ref.egs_rho_cut(rth) == pytest.approx(p["egs_cut"], abs=1e-15)
    # Proposition 4.3: with rho_oo = lambda the lower bound of rho_hat_to is rho_th
    assert float(ref.transitive_lower(rmax, ref.lam(rth, rmax))) == pytest.approx(rth, abs=1e-12)


# ---------------------------------------------------------------------------
# Group layout
# ---------------------------------------------------------------------------
def _centres_by_enumeration(length, h):
    out = []
    members = list(range(length))
    for g in range(0, length, h):
        grp = members[g:g + h]
        out.append(sorted(grp)[(len(grp) - 1) // 2])
    return out


@pytest.mark.parametrize("length,h", [(1, 1), (10, 3), (11, 3), (241, 3), (100, 7), (13, 9), (4, 9)])
def test_group_centres(length, h):
    exp = _centres_by_enumeration(length, h)
    assert list(ref.group_centres_axis(length, h)) == exp
    for c in range(length):
        assert ref.group_centre(c, length, h) == exp[c // h]
    assert ref.n_groups(length, 5, h) == len(exp) * len(_centres_by_enumeration(5, h))


# ---------------------------------------------------------------------------
# Section 4 blur, Algorithm 3 blur correlation, Algorithm 1 auto-correlation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("s", [0.5, 1.0, 2.0, 3.0])
def test_uniform_blur_equals_library_gaussian(s):
    from scipy import ndimage
    img = synth.white_blur_image(70, seed=8)
    out = ref.blur(img, np.full((2, 2), s), 64)
    # scipy's truncate=3 radius int(3 s + 0.5) equals ceil(3 s) at these sigmas
    exp = ndimage.gaussian_filter(img.astype(np.float64), s, mode="nearest", truncate=3.0)
    assert np.allclose(out, exp, atol=1e-10)


def test_blur_block_map_and_identity():
    from scipy import ndimage
    img = synth.white_blur_image(100, seed=9)
    smap = np.array([[0.0, 2.0], [1.0, 0.5]])
    out = ref.blur(img, smap, 64)
    for by in range(2):
        for bx in range(2):
            ys = slice(by * 64, min(100, by * 64 + 64)); xs = slice(bx * 64, min(100, bx * 64 + 64))
            s = smap[by, bx]
            exp = img if s == 0 else ndimage.gaussian_filter(img.astype(float), s, mode="nearest", truncate=3.0)
            assert np.allclose(out[ys, xs], exp[ys, xs], atol=1e-10)
    const = np.full((30, 30), 77.0)
    assert np.allclose(ref.blur(const, np.full((1, 1), 3.0), 64), 77.0, atol=1e-12)


def test_blur_corr_map():
    img = synth.white_blur_image(50, seed=14)
    m, n = 6, 9
    R0 = ref.blur_corr_map(img, img, m, n)
    assert np.allclose(R0, 1.0, atol=1e-12)
    P = ref.quantise_pivot(ref.blur(img, np.full((1, 1), 1.0), 64))
    R = ref.blur_corr_map(P, img, m, n)
    for (y, x) in [(0, 0), (10, 20), (44, 41)]:
        a = P[y:y + m, x:x + n].astype(float).ravel(); b = img[y:y + m, x:x + n].ravel()
        assert R[y, x] == pytest.approx(np.corrcoef(a, b)[0, 1], abs=1e-12)


def test_rho_co_map():
    img = synth.white_blur_image(60, seed=15)
    m, n, h = 7, 5, 3
    Ly, Lx = 60 - m + 1, 60 - n + 1
    P = ref.quantise_pivot(ref.blur(img, np.full((1, 1), 2.0), 64))
    R = ref.rho_co_map(P, img, m, n, h)
    cy = _centres_by_enumeration(Ly, h); cx = _centres_by_enumeration(Lx, h)
    rng = np.random.default_rng(0)
    for _ in range(40):
        y = int(rng.integers(0, Ly)); x = int(rng.integers(0, Lx))
        c = P[cy[y // h]:cy[y // h] + m, cx[x // h]:cx[x // h] + n].astype(float).ravel()
        o = img[y:y + m, x:x + n].ravel()
        assert R[y, x] == pytest.approx(np.corrcoef(c, o)[0, 1], abs=1e-12)
    # unblurred pivot: the centres correlate perfectly with themselves
    R1 = ref.rho_co_map(img, img, m, n, h)
    assert np.allclose(R1[np.ix_(cy, cx)], 1.0, atol=1e-12)
    # h = 1 is the blur correlation map
    assert np.allclose(ref.rho_co_map(P, img, m, n, 1), ref.blur_corr_map(P, img, m, n), atol=0)


# ---------------------------------------------------------------------------
# Section 3: EGS
# ---------------------------------------------------------------------------
def test_egs_cost_counts():
    rco = np.array([[0.9, 0.59, 0.6], [0.61, -0.2, 0.95]])
    # groups of h=3 over a 2 x 3 location grid -> 1 group; retained: 0.59 and -0.2
    assert ref.egs_cost(rco, 3, 0.8) == 1 + 2
    assert ref.egs_cost(rco, 1, 0.8) == 6 + 2


@pytest.mark.parametrize("Ly,h,sample", [(100, 1, 4), (241, 3, 4), (4033, 5, 4), (40, 9, 2), (7, 3, 4)])
def test_egs_sample_rows_by_enumeration(Ly, h, sample):
    """The sampled rows: group rows in runs of 8, every sample-th run (and
    all rows of a group row, including the short last group)."""
    want = np.zeros(Ly, dtype=bool)
    groups = [list(range(g, min(g + h, Ly))) for g in range(0, Ly, h)]
    for gi, rows in enumerate(groups):
        if (gi // 8) % sample == 0:
            want[rows] = True
    assert np.array_equal(ref.egs_sample_rows(Ly, h, sample), want)
    assert ref.egs_sample_rows(Ly, h, 1).all()


def test_egs_sampled_cost_scales_the_sampled_count():
    Ly, Lx, h = 96, 10, 3             # 32 group rows: runs 0..3, run 0 sampled (rows 0..23)
    rco = np.ones((Ly, Lx))
    rco[0:6, :4] = 0.0                # 24 retained inside the sample
    rco[30:40, :] = 0.0               # 100 retained outside it
    groups = 32 * 4
    assert ref.egs_cost(rco, h, 0.8, sample=1) == groups + 124
    # sampled rows 0..23 hold 24 retained: 24 * 96 / 24 = 96
    assert ref.egs_cost(rco, h, 0.8, sample=4) == groups + 96
    # rounding to nearest: 1 retained over 24 sampled rows of 96 -> 4
    one = np.ones((Ly, Lx)); one[5, 5] = 0.0
    assert ref.egs_cost(one, h, 0.8, sample=4) == groups + 4


def test_egs_stop_rule(monkeypatch):
    """Algorithm 2 grows h while the cost drops by more than xi of the last cost."""
    costs = {1: 1000, 3: 500, 5: 498, 7: 100, 9: 100}
    monkeypatch.setattr(ref, "rho_co_map", lambda P, I, m, n, h, threads=0: h)
    monkeypatch.setattr(ref, "egs_cost", lambda r, h, rho_th, sample=1: costs[h])
    log = []
    assert ref.egs(None, None, 4, 4, 1, 0.8, 0.005, log=log) == (3, 500)
    assert log == [(1, 1000), (3, 500), (5, 498)]
    assert ref.egs(None, None, 4, 4, 1, 0.8, 0.0) == (7, 100)
    assert ref.egs(None, None, 4, 4, 7, 0.8, 0.005, h_max=7) == (7, 100)


def test_opta_invariants():
    img = synth.aerial_image(256, n_octaves=6, n_prims=12, seed=77).astype(np.float64)
    res = ref.opta(img, 16, 16)
    tr = res["trace"]
    kept = [tr[0]]
    for a in tr[1:]:
        if kept[-1]["cost"] - a["cost"] > 0.005 * kept[-1]["cost"]:
            kept.append(a)
        else:
            break
    assert res["cost"] == kept[-1]["cost"] and res["h"] == kept[-1]["h"]
    assert set(np.unique(res["sigma_map"])) <= {0.0, 0.5, 1.0, 2.0, 3.0}
    assert res["pivot"].dtype == np.uint8
    # rho_max = rho_th gives lambda = 1: no block may ever be blurred
    res1 = ref.opta(img, 16, 16, rho_th=0.8, rho_max=0.8)
    assert np.all(res1["sigma_map"] == 0.0)


# ---------------------------------------------------------------------------
# Section 4.3: search on the blurred image, local re-match on I
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("s,d", [(0.0, 0), (0.5, 2), (1.0, 3), (2.0, 6), (3.0, 9)])
def test_literal_support_is_filter_half_width(s, d):
    smap = np.array([[0.0, s], [0.0, 0.0]])
    assert ref.literal_support(smap) == d


def test_literal_search_reduces_to_exact_search():
    img = synth.aerial_image(96, n_octaves=5, n_prims=8, seed=21).astype(np.float64)
    t = img[30:42, 50:61] + np.random.default_rng(2).normal(0, 3.0, (12, 11))
    y, x, r = ref.best_match(img, t)
    # no blur and no neighbourhood: the search on P = I is the exact search
    assert ref.literal_search(img, ref.quantise_pivot(img), t, 0)[:3] == (y, x, r)
    # a neighbourhood covering every location: exact whatever P is
    P = ref.quantise_pivot(ref.blur(img, np.full((2, 2), 3.0), 64))
    Ly, Lx = img.shape[0] - 11, img.shape[1] - 10
    assert ref.literal_search(img, P, t, max(Ly, Lx))[:3] == (y, x, r)


def test_literal_search_stays_in_the_neighbourhood():
    img = synth.aerial_image(96, n_octaves=5, n_prims=8, seed=22).astype(np.float64)
    P = ref.quantise_pivot(ref.blur(img, np.full((2, 2), 2.0), 64))
    t = img[60:76, 10:26].copy()
    y, x, r, yh, xh = ref.literal_search(img, P, t, 3)
    # (y_hat, x_hat) is the exact maximum on P; (y, x) the best of I within d
    assert (yh, xh) == ref.best_match(P, t)[:2]
    assert abs(y - yh) <= 3 and abs(x - xh) <= 3
    assert r == ref.rho_at(img, t, [y], [x])[0]
    ys, xs = np.meshgrid(np.arange(max(0, yh - 3), yh + 4), np.arange(max(0, xh - 3), xh + 4), indexing="ij")
    assert r >= ref.rho_at(img, t, ys.ravel(), xs.ravel()).max()


def test_opta_literal_measures_the_pivot_auto_correlation(monkeypatch):
    """EGS in the literal mode receives the candidate pivot on both sides."""
    img = synth.aerial_image(128, n_octaves=5, n_prims=8, seed=23).astype(np.float64)
    seen = []
    real = ref.egs

    def spy(P, I, *a, **k):
        seen.append((P, I))
        return real(P, I, *a, **k)

    monkeypatch.setattr(ref, "egs", spy)
    res = ref.opta_literal(img, 16, 16)
    assert len(seen) >= 2 and all(a is b for a, b in seen)
    assert res["pivot"].dtype == np.uint8
    seen.clear()
    ref.opta(img, 16, 16)
    assert all(b is not a for a, b in seen[1:])


def test_opta_literal_without_blur_is_opta():
    """lambda = 1 forbids every blur, so P = I and both modes measure rho(I, I)."""
    img = synth.aerial_image(128, n_octaves=5, n_prims=8, seed=24).astype(np.float64)
    a = ref.opta_literal(img, 16, 16, rho_th=0.8, rho_max=0.8)
    b = ref.opta(img, 16, 16, rho_th=0.8, rho_max=0.8)
    assert np.all(a["sigma_map"] == 0) and a["h"] == b["h"] and a["cost"] == b["cost"]


# ---------------------------------------------------------------------------
# Algorithm 3: which block a failing window freezes
# ---------------------------------------------------------------------------
def test_opta_freezes_the_block_of_the_failing_windows_top_left():
    """A non-square image (3 x 4 blocks of 64) that is a linear ramp except
    for one 8 x 8 patch of white noise.  Blurring a ramp changes it by less
    than rounding, so only windows that reach the patch's blurred support can
    fall below lambda (Eq. misDec): at sigma = 1 the blurred noise keeps a
    correlation of about 0.56 with itself.  The patch sits where every such
    window has its top-left corner in block (1, 3), while the bottom-right
    corners of some lie in block (2, 3); so exactly block (1, 3) must fail
    and freeze -- a swapped (row, column) block index or a window assigned
    by another corner fails this."""
    p, q = 192, 256
    yy, xx = np.mgrid[0:p, 0:q]
    img = np.rint(0.6 * yy + 0.45 * xx)
    img[115:123, 226:234] = np.random.default_rng(5).integers(0, 256, (8, 8))
    res = ref.opta(img, 8, 8, levels=(1.0,))
    lvl = res["trace"][1]
    want = np.zeros((3, 4), dtype=bool)
    want[1, 3] = True
    assert lvl["fail"].shape == (3, 4)
    assert np.array_equal(lvl["fail"], want)
    assert np.array_equal(lvl["frozen_map"], want)
    assert lvl["frozen"] == 1
    # the same ramp without the patch: nothing fails
    clean = ref.opta(np.rint(0.6 * yy + 0.45 * xx), 8, 8, levels=(1.0,))
    assert not clean["trace"][1]["fail"].any()
    # a frozen block keeps its previous sigma: with a second level the
    # patch's block stays at 0 wherever the loop stops
    two = ref.opta(img, 8, 8, levels=(1.0, 2.0), xi=-1.0)   # accept every level
    assert two["sigma_map"][1, 3] == 0.0
    assert np.all(np.delete(two["sigma_map"].ravel(), 1 * 4 + 3) > 0.0)


def test_quantise_pivot_rounds_half_to_even_and_clips():
    got = ref.quantise_pivot(np.array([[0.5, 1.5, 2.5, -3.0], [300.0, 254.5, 254.49, 7.5]]))
    assert got.dtype == np.uint8
    assert got.tolist() == [[0, 2, 2, 0], [255, 254, 254, 8]]


# ---------------------------------------------------------------------------
# The FFT form of Eq. rho1 against the direct definition
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,tshape,seed", [
    ((61, 47), (9, 13), 1),        # ragged sizes
    ((40, 40), (40, 40), 2),       # one location (template = image size)
    ((33, 70), (1, 7), 3),         # one-row template
    ((50, 64), (16, 16), 4),
])
def test_fft_map_equals_direct_definition(shape, tshape, seed):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, size=shape).astype(np.float64)
    img[5:25, 3:30] = 200.0                                   # flat windows
    t = rng.normal(100.0, 30.0, size=tshape)
    a = ref.zncc_map(img, t)
    b = ref.zncc_map_fft(img, t)
    assert b.shape == a.shape
    assert np.max(np.abs(a - b)) < 1e-12
    assert np.array_equal(a == 0.0, b == 0.0) or np.all(np.abs(b[a == 0.0]) < 1e-12)


def test_fft_map_non_integer_image_and_flat_template():
    rng = np.random.default_rng(6)
    img = rng.normal(size=(45, 52))
    t = rng.normal(size=(7, 11))
    assert np.max(np.abs(ref.zncc_map(img, t) - ref.zncc_map_fft(img, t))) < 1e-12
    assert np.all(ref.zncc_map_fft(img, np.full((7, 11), 3.0)) == 0.0)


def test_fft_map_exact_crop_and_affine_template():
    img = synth.aerial_image(160, n_octaves=6, n_prims=8, seed=17)
    t = 1.3 * img[40:72, 90:122].astype(np.float64) - 17.0
    rho = ref.zncc_map_fft(img, t)
    assert abs(rho[40, 90] - 1.0) < 1e-12
    assert ref.argmax_first(rho)[:2] == (40, 90)
